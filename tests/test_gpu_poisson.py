"""The embedded-boundary Poisson solve on the GPU (conjugate gradients on -C,
Sec. 2; the virus-shaped domain of Sec. 4.1) against the oracle's direct
solve, the exact solution of affine data, and second-order convergence."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import poisson  # noqa: E402
from oracle.eb import EBOperator  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from paper_2209_15095_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    return etd


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _gpu_solve(lib, w, beta_field, u_gamma, f_grid, tol=1e-13):
    ctx = lib.Context(w.n, w.lo, w.hi, precision="fp64", tol=1e-10, m_max=30, reaction="none", mu=(0.0,),
                      beta=(1.0,), boundary_data=True)
    ctx.init_domain(0, _dev(w.phi0[0]), None if beta_field is None else _dev(beta_field))
    P = ctx.boundary_points(0).cpu().numpy()
    vals = _dev(u_gamma(P))
    ctx.set_boundary_values(0, vals)
    u = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    it, res = ctx.poisson_solve(0, _dev(f_grid), u, tol=tol, max_iter=50000)
    assert res <= tol
    return u.cpu().numpy(), it


def test_poisson_matches_direct_solve(lib):
    w = inputs.virus2d(100)
    g = Grid(w.n, w.lo, w.hi)
    op = EBOperator(g, w.phi0[0], w.beta_field, boundary_data=True)
    ug = lambda P: inputs.virus_exact(P[..., 0], P[..., 1])
    uo = poisson.solve(op, op.from_grid(w.source), ug)
    u, it = _gpu_solve(lib, w, w.beta_field, ug, w.source)
    assert it > 10
    assert np.max(np.abs(op.from_grid(u) - uo)) <= 1e-9 * np.max(np.abs(uo))


def test_poisson_affine_exact(lib):
    w = inputs.virus2d(200)
    g = Grid(w.n, w.lo, w.hi)
    op = EBOperator(g, w.phi0[0], 1.0, boundary_data=True)
    assert op.nclamp == 0
    ua = lambda P: 1.0 + 2.0 * P[..., 0] - 3.0 * P[..., 1]
    u, _ = _gpu_solve(lib, w, None, ua, np.zeros(w.n))
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    assert np.max(np.abs(op.from_grid(u) - ua(X))) < 1e-8


def test_poisson_second_order_on_gpu(lib):
    errs = []
    for N in (50, 100, 200):
        w = inputs.virus2d(N)
        g = Grid(w.n, w.lo, w.hi)
        op = EBOperator(g, w.phi0[0], w.beta_field, boundary_data=True)
        ug = lambda P: inputs.virus_exact(P[..., 0], P[..., 1])
        u, _ = _gpu_solve(lib, w, w.beta_field, ug, w.source)
        X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
        e = op.from_grid(u) - inputs.virus_exact(X[:, 0], X[:, 1])
        errs.append((np.max(np.abs(e)), math.sqrt(np.mean(e * e))))
    for j in range(2):
        orders = [math.log2(errs[i][j] / errs[i + 1][j]) for i in range(2)]
        assert min(orders) > 1.6, (errs, orders)
