"""ETD3RK and ETD4RK on the GPU (Sec. 3.2) and the phi-combination with p = 3
(Eq. 3.9) through the C ABI, against the FP64 oracle.

1e-10 relative (FP64): the p = 3 combination and two steps of each scheme
from identical inputs, the oracle replaying the GPU's decision trace (per
stage for the Runge-Kutta schemes); 1e-5 relative for the FP32-mixed path
against the oracle at tolerance 1e-12.  Two species coupled through the competition
reaction, and temporal order 4 of ETD4RK on a stiff EB system against a
tight explicit reference.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etd as oetd  # noqa: E402
from oracle import krylov  # noqa: E402
from oracle.eb import EBOperator  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from _replay import forced, split_evaluations  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    return etd


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ellipsoid(ndim, n, box):
    g = Grid((n,) * ndim, (-box,) * ndim, (box,) * ndim)
    x = g.coords()
    a = [0.7, 0.55, 0.5, 0.45][:ndim]
    return g, np.sqrt(sum((x[d] / (a[d] * box)) ** 2 for d in range(ndim))) - 1.0


def _ball(ndim, n, box, R):
    g = Grid((n,) * ndim, (-box,) * ndim, (box,) * ndim)
    return g, np.sqrt(sum(c * c for c in g.coords())) - R


def _ctx(lib, g, **kw):
    args = dict(nspecies=1, precision="fp64", tol=1e-10, m_max=40, reaction="logistic", mu=(1.0,), beta=(1.0,))
    args.update(kw)
    return lib.Context(g.n, g.lo, g.hi, **args)


def _phipm_replayed(op, dt, vs, tol, m_max, stats):
    """The oracle's combination; if its decisions differ from the GPU's trace,
    the oracle replays the GPU's (tau, m) sequence."""
    apply_A = lambda x: dt * (op.C @ x)
    anorm = dt * op.gershgorin()
    yo, tr = krylov.phipm(apply_A, vs, tol, m_max, anorm)
    gtr = list(stats["trace"])
    if [m for _, m in gtr] != [m for _, m, _ in tr] or len(gtr) != len(tr):
        yo, tr = krylov.phipm(apply_A, vs, tol, m_max, anorm, forced_trace=[(t, m, 0) for t, m in gtr])
    return yo, tr


@pytest.mark.parametrize("ndim,n,box,shape", [(2, 40, 1.0, "ellipsoid"), (3, 22, 2.0, "ellipsoid"),
                                               (4, 13, 2.0, "ball")])
def test_phi_combination3_fp64(lib, ndim, n, box, shape):
    g, ph = _ellipsoid(ndim, n, box) if shape == "ellipsoid" else _ball(ndim, n, box, 0.62 * box)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(31 + n)
    vs = [rng.standard_normal(op.ncomp) for _ in range(4)]
    dt = 0.8 * g.h
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination3(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    yg = op.from_grid(y.cpu().numpy())
    yo, tr = _phipm_replayed(op, dt, vs, 1e-10, 40, st)
    assert np.max(np.abs(yg - yo)) <= 1e-10 * np.max(np.abs(yo)), (st, tr)
    assert np.all(y.cpu().numpy()[~op.comp] == 0.0)


def test_phi_combination3_reduces_to_p2(lib):
    # v3 = 0: the p = 3 combination equals the p = 2 one (a different substep
    # recursion and error estimate, the same sum)
    g, ph = _ellipsoid(3, 22, 2.0)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, tol=1e-12)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(5)
    vs = [_dev(op.to_grid(rng.standard_normal(op.ncomp))) for _ in range(3)]
    y2 = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    y3 = torch.zeros_like(y2)
    dt = 0.5 * g.h
    ctx.phi_combination(0, dt, *vs, y2)
    ctx.phi_combination3(0, dt, *vs, torch.zeros_like(y2), y3)
    ctx.sync()
    assert torch.max(torch.abs(y3 - y2)).item() <= 1e-10 * torch.max(torch.abs(y2)).item()


@pytest.mark.parametrize("precision,n,split_min", [("fp64", 112, 1 << 17), ("mixed", 140, 1 << 18)])
def test_phi_combination3_large_split_pass(lib, precision, n, split_min):
    """Above the split-pass threshold (2^17 FP64, 2^18 FP32 points)."""
    g, ph = _ball(3, n, 2.0, 1.24)
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp >= split_min
    tol = 1e-10 if precision == "fp64" else 1e-7
    ctx = _ctx(lib, g, precision=precision, tol=tol)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(19)
    u = rng.uniform(0, 1, op.ncomp)
    # |dt C| about 4N, the stiffness of the workloads.  FP32 rounding of w_2
    # (about eps_32 |A| |w_1|) enters y through tau^2 phi_2(tau A), so the
    # mixed path's error on rough data grows with |dt C|^2: at dt = 2 h^2 it
    # was 4.5e-5 relative.
    dt = g.h * g.h
    F = u * (1 - u)
    vs = [u, dt * F, 0.3 * dt * F, -0.2 * dt * F]
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination3(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    yg = op.from_grid(y.cpu().numpy())
    if precision == "fp64":
        yo, tr = _phipm_replayed(op, dt, vs, tol, 40, st)
        assert np.max(np.abs(yg - yo)) <= 1e-10 * np.max(np.abs(yo)), (st, tr)
    else:
        yo, _ = krylov.phipm(lambda x: dt * (op.C @ x), vs, 1e-12, 40, dt * op.gershgorin())
        assert np.max(np.abs(yg - yo)) <= 1e-5 * np.max(np.abs(yo))


@pytest.mark.parametrize("scheme", ["etd3rk", "etd4rk"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_etd3rk_etd4rk_steps(lib, scheme, precision, tol):
    """Two steps through etd_step against the oracle's stages; the statistics
    add the three or four evaluations of a step."""
    g, ph = _ellipsoid(3, 26, 2.0)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, precision=precision, tol=1e-10 if precision == "fp64" else 1e-6, scheme=scheme)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(9)
    u0 = op.to_grid(rng.uniform(0, 1, op.ncomp))
    du = _dev(u0)
    dt = 0.02
    step = oetd.etd3rk_step if scheme == "etd3rk" else oetd.etd4rk_step
    nev = 3 if scheme == "etd3rk" else 4
    F_of = lambda v, t: v * (1 - v)
    uo = op.from_grid(u0)
    fp64 = precision == "fp64"
    for _ in range(2):
        st = ctx.step(dt, [du], stats=True)[0]
        assert st["substeps"] >= nev and len(st["trace"]) == st["substeps"]
        # FP64: the oracle at the GPU's tolerance replays each stage's
        # decisions; mixed: against the oracle at 1e-12
        fts = split_evaluations(st["trace"], nev) if fp64 else None
        uo, _, traces = step(op, uo, F_of, 0.0, dt, tol=1e-10 if fp64 else 1e-12, m_max=40, forced_traces=fts)
        ug = du.cpu().numpy()
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= tol * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)


class _BlockOp:
    """Two species' operators as one block-diagonal system (oracle side)."""

    def __init__(self, ops):
        import scipy.sparse as sp

        self.ops = ops
        self.C = sp.block_diag([o.C for o in ops]).tocsr()
        self.ncomp = sum(o.ncomp for o in ops)

    def gershgorin(self):
        return max(o.gershgorin() for o in self.ops)

    def split(self, u):
        n0 = self.ops[0].ncomp
        return u[:n0], u[n0:]


def test_etd4rk_two_species_competition(lib):
    # overlapping discs: each species' F reads the other's stage value where
    # that point is computational for the other species, else 0
    n = 48
    g = Grid((n, n), (-2.0, -2.0), (2.0, 2.0))
    x, y = g.coords()
    phs = [np.sqrt((x + 0.45) ** 2 + y ** 2) - 1.1, np.sqrt((x - 0.45) ** 2 + y ** 2) - 1.0]
    beta, rp = (1.0, 0.7), (0.5, 0.8, 1.2)
    ops = [EBOperator(g, phs[s], beta[s]) for s in range(2)]
    blk = _BlockOp(ops)
    cross = [ops[0].from_grid(ops[1].comp.astype(float)), ops[1].from_grid(ops[0].comp.astype(float))]
    assert min(c.sum() for c in cross) > 50  # the domains overlap

    def F_of(u, t):
        u0, u1 = blk.split(u)
        v_at0 = ops[0].from_grid(ops[1].to_grid(u1))
        u_at1 = ops[1].from_grid(ops[0].to_grid(u0))
        a, b, r = rp
        return np.concatenate([u0 * (1 - u0 - a * v_at0), r * u1 * (1 - u1 - b * u_at1)])

    rng = np.random.default_rng(4)
    us = [rng.uniform(0.2, 0.9, o.ncomp) for o in ops]
    ctx = lib.Context(g.n, g.lo, g.hi, nspecies=2, precision="fp64", tol=1e-10, m_max=40, reaction="competition",
                      rparams=rp, mu=(1.0, 1.0), beta=beta, scheme="etd4rk")
    du = [_dev(ops[s].to_grid(us[s])) for s in range(2)]
    for s in range(2):
        ctx.init_domain(s, _dev(phs[s]))
    uo = np.concatenate(us)
    dt = 0.01
    for _ in range(2):
        ctx.step(dt, du)
        uo, _, _ = oetd.etd4rk_step(blk, uo, F_of, 0.0, dt, tol=1e-12, m_max=40)
        for s, us_o in enumerate(blk.split(uo)):
            ug = ops[s].from_grid(du[s].cpu().numpy())
            assert np.max(np.abs(ug - us_o)) <= 1e-9 * np.max(np.abs(us_o))


def test_etd4rk_temporal_order_on_gpu(lib):
    # The stiff EB system of the oracle's order pin (a disc, spectral radius
    # about 108, logistic reaction) stepped on the GPU: order 4 against
    # scipy's DOP853, and parity with the oracle's dense-expm stages.
    from scipy.integrate import solve_ivp

    g = Grid((16, 16), (-2, -2), (2, 2))
    ph = g.radius() - 1.3
    op = EBOperator(g, ph, 1.0)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    u0 = 0.5 + 0.4 * np.cos(X[:, 0]) * np.sin(X[:, 1] + 0.3)
    F_of = lambda u, t: u * (1.0 - u)
    C = op.C.toarray()
    T = 0.8
    ref = solve_ivp(lambda t, u: C @ u + F_of(u, t), (0.0, T), u0, method="DOP853", rtol=3e-14,
                    atol=1e-15).y[:, -1]
    ctx = _ctx(lib, g, tol=1e-12, scheme="etd4rk")
    ctx.init_domain(0, _dev(ph))
    errs = []
    for nst in (16, 32, 64):
        du = _dev(op.to_grid(u0))
        for _ in range(nst):
            ctx.step(T / nst, [du])
        ug = op.from_grid(du.cpu().numpy())
        errs.append(np.max(np.abs(ug - ref)))
        if nst == 16:
            uo = oetd.run_fixed_domain(op, u0, T / nst, nst, F_of, exact=True, scheme="etd4rk")
            assert np.max(np.abs(ug - uo)) <= 1e-10 * np.max(np.abs(uo))
    assert math.log2(errs[1] / errs[2]) > 3.5, errs


def test_rk34_argument_checks(lib):
    g, ph = _ellipsoid(2, 24, 1.0)
    with pytest.raises(lib.EtdError):
        _ctx(lib, g, m_max=61, scheme="etd3rk")
    ctx = _ctx(lib, g, m_max=61)
    ctx.init_domain(0, _dev(ph))
    z = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.EtdError):
        ctx.phi_combination3(0, 0.01, z, z, z, z, torch.zeros_like(z))
    ctx = _ctx(lib, g, scheme="etd4rk")
    ctx.init_domain(0, _dev(ph))
    ctx.set_source(0, torch.ones_like(z))
    with pytest.raises(lib.EtdError):
        ctx.step(0.01, [torch.zeros_like(z)])


def _oracle_etd3(op, uo, hist, F_n, dt, tol=1e-12, ft=None):
    """One step of the oracle's multistep ETD3 with the start-up reading
    (ft: a decision trace to replay).  The GPU evaluates the start-up steps
    (ETD1, ETD2) as p = 3 combinations with v_3 = 0; a replayed trace needs
    the same Krylov vector w_3, so the replayed start-up uses that form too
    (the same phi-combination, Eq. 3.9)."""
    hist.insert(0, F_n)
    del hist[3:]
    if len(hist) == 3:
        return oetd.etd3_step(op, uo, hist[0], hist[1], hist[2], dt, tol=tol, m_max=40, forced_trace=ft)[0]
    if ft is not None:
        vs = oetd.etd2_vectors(uo, hist[0], hist[-1], dt) + [np.zeros_like(uo)]
        return oetd.combination(op, vs, dt, tol=tol, m_max=40, forced_trace=ft)[0]
    return oetd.etd2_step(op, uo, hist[0], hist[-1], dt, tol=tol, m_max=40, forced_trace=ft)[0]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_etd3_multistep_steps(lib, precision, tol):
    """Four multistep ETD3 steps (Eq. 3.8b, s = 3) through etd_step: ETD1, ETD2,
    then ETD3 from the stored F_{n-1}, F_{n-2}, against the oracle."""
    g, ph = _ellipsoid(3, 26, 2.0)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, precision=precision, tol=1e-10 if precision == "fp64" else 1e-6, scheme="etd3")
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(12)
    u0 = op.to_grid(rng.uniform(0, 1, op.ncomp))
    du = _dev(u0)
    dt = 0.02
    uo, hist = op.from_grid(u0), []
    fp64 = precision == "fp64"
    for _ in range(4):
        st = ctx.step(dt, [du], stats=True)[0]
        if fp64:
            uo = _oracle_etd3(op, uo, hist, uo * (1 - uo), dt, tol=1e-10, ft=forced(st["trace"]))
        else:
            uo = _oracle_etd3(op, uo, hist, uo * (1 - uo), dt)
        ug = du.cpu().numpy()
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= tol * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)


def test_etd3_multistep_with_boundary_data(lib):
    """ETD3 on the peanut problem of Table 1 (Sec. 4.2.1): a source and nonzero
    Dirichlet data enter F and the stored history; three steps against the
    oracle with the same readings."""
    n = 61
    g = Grid((n, n), (-1.0, -1.0), (1.0, 1.0))
    x, y = g.coords()
    rho = 0.5 - np.exp(-20 * (x ** 2 + (y - 0.25) ** 2)) - np.exp(-20 * (x ** 2 + (y + 0.25) ** 2))
    beta = 0.25 - x ** 2 - y ** 2
    r2 = x ** 2 + y ** 2
    op = EBOperator(g, rho, beta, boundary_data=True)
    ctx = lib.Context(g.n, g.lo, g.hi, precision="fp64", tol=1e-12, m_max=40, reaction="none", mu=(0.0,),
                      beta=(1.0,), boundary_data=True, scheme="etd3")
    ctx.init_domain(0, _dev(rho), _dev(beta))
    P = ctx.boundary_points(0).cpu().numpy()
    u_gamma = lambda Q, t: np.exp(-t) * (np.sum(Q ** 2, axis=-1) - 0.25)
    source = lambda rr, t: math.exp(-t) * (28 * rr - 3) / 4
    rc = op.from_grid(r2)
    du = _dev(op.to_grid(rc - 0.25))
    uo, hist, t, dt = rc - 0.25, [], 0.0, g.h
    keep = []
    for _ in range(3):
        vals, src = _dev(u_gamma(P, t)), _dev(source(r2, t))
        keep.append((vals, src))  # the library reads them during the step
        ctx.set_boundary_values(0, vals)
        ctx.set_source(0, src)
        ctx.step(dt, [du])
        F_n = source(rc, t) + op.boundary_rhs(lambda Q: u_gamma(Q, t))
        uo = _oracle_etd3(op, uo, hist, F_n, dt)
        t += dt
        ug = op.from_grid(du.cpu().numpy())
        assert np.max(np.abs(ug - uo)) <= 1e-10 * np.max(np.abs(uo))
