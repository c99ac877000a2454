"""Adjoint path on the GPU (through the C ABI): the explicit ETD2 step and
one adjoint step against the FP64 oracle (1e-10 relative in FP64, 1e-5 in
FP32-mixed), and the gradients of a terminal loss through the torch.autograd
wrapper against central finite differences of the FP64 GPU forward (1e-4
relative) and against the oracle's adjoint gradient (1e-10 relative in FP64,
1e-4 in FP32-mixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj  # noqa: E402
from oracle.eb import EBOperator  # noqa: E402
from oracle.grid import Grid  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    return etd


def _case(ndim=3, n=18, R=1.0, seed=0):
    g = Grid((n,) * ndim, (-1.6,) * ndim, (1.6,) * ndim)
    x = g.coords()
    r = np.sqrt(sum(c * c for c in x))
    ph = r - R
    beta = 1.0 + 0.3 * np.sin(1.7 * x[0] + 0.4) * np.cos(1.1 * x[1])
    op = EBOperator(g, ph, beta)
    rng = np.random.default_rng(seed)
    return g, ph, beta, op, rng


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ctx(lib, g, alpha=1.0, K=1.0, tol=1e-12, precision="fp64"):
    return lib.Context(g.n, g.lo, g.hi, nspecies=1, precision=precision, tol=tol, m_max=40, reaction="logistic_ak",
                       rparams=(alpha, K), adjoint=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_explicit_step_and_adjoint_step(lib, precision):
    g, ph, beta, op, rng = _case()
    alpha, K, dt, nq = 1.1, 1.0, 0.03, 8
    fp64 = precision == "fp64"
    bound = 1e-10 if fp64 else 1e-5
    ctx = _ctx(lib, g, alpha, K, tol=1e-12 if fp64 else 1e-8, precision=precision)
    dbeta = _dev(beta)
    ctx.init_domain(0, _dev(ph), dbeta)
    u_n = op.to_grid(rng.uniform(0.2, 0.9, op.ncomp))
    u_nm1 = op.to_grid(rng.uniform(0.2, 0.9, op.ncomp))
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ctx.step_explicit(0, dt, _dev(u_n), _dev(u_nm1), out)
    pe = oadj.PhiEval(op, exact=True)
    un_c, unm1_c = op.from_grid(u_n), op.from_grid(u_nm1)
    F = oadj.reaction_ak(un_c, alpha, K)
    Fm = oadj.reaction_ak(unm1_c, alpha, K)
    ref = pe.comb(dt, [un_c, dt * F, dt * (F - Fm)])
    got = op.from_grid(out.cpu().numpy())
    assert np.max(np.abs(got - ref)) <= bound * np.max(np.abs(ref))
    # one adjoint step
    lam = op.to_grid(rng.standard_normal(op.ncomp))
    acc0 = op.to_grid(rng.standard_normal(op.ncomp))
    dl, da = _dev(lam), _dev(acc0)
    gb = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.adjoint_step(0, dt, _dev(u_n), _dev(u_nm1), False, dl, da, gb, ga, nq)
    ctx.sync()
    # the oracle evaluates every phi action exactly (dense augmented expm)
    to_n, to_nm1, dalpha, dbeta_o = oadj.adjoint_step(op, pe, dt, un_c, unm1_c, op.from_grid(lam), alpha, K, nq)
    lam_ref = to_n + op.from_grid(acc0)
    assert np.max(np.abs(op.from_grid(dl.cpu().numpy()) - lam_ref)) <= bound * np.max(np.abs(lam_ref))
    assert np.max(np.abs(op.from_grid(da.cpu().numpy()) - to_nm1)) <= bound * np.max(np.abs(to_nm1))
    assert abs(ga.item() - dalpha) <= bound * abs(dalpha)
    gbo = dbeta_o.ravel()
    assert np.max(np.abs(gb.cpu().numpy().ravel() - gbo)) <= bound * np.max(np.abs(gbo))


def test_trajectory_gradients(lib):
    from paper_2209_15095_gb300.autograd import trajectory

    g, ph, beta, op, rng = _case(n=16, seed=3)
    alpha0, K, dt, nsteps, every, nq = 1.0, 1.0, 0.02, 7, 3, 10
    ctx = _ctx(lib, g, alpha0, K)
    dph = _dev(ph)
    u0 = op.to_grid(rng.uniform(0.2, 0.9, op.ncomp))
    target = op.to_grid(rng.uniform(0.0, 0.5, op.ncomp))
    du0 = _dev(u0).requires_grad_(True)
    dbeta = _dev(beta).requires_grad_(True)
    dalpha = torch.tensor([alpha0], dtype=torch.float64, device="cuda", requires_grad=True)
    dtarget = _dev(target)
    uT = trajectory(ctx, du0, dbeta, dalpha, dph, dt, nsteps, K=K, checkpoint_every=every, nquad=nq)
    loss = 0.5 * ((uT - dtarget) ** 2).sum()
    loss.backward()
    gu, gb, ga = du0.grad.cpu().numpy(), dbeta.grad.cpu().numpy(), dalpha.grad.item()

    def L(u0_, beta_, alpha_):
        with torch.no_grad():
            out = trajectory(ctx, _dev(u0_), _dev(beta_), torch.tensor([alpha_], dtype=torch.float64, device="cuda"),
                             dph, dt, nsteps, K=K, checkpoint_every=every, nquad=nq)
            return 0.5 * float(((out - dtarget) ** 2).sum())

    eps = 1e-6
    comp = np.flatnonzero(op.comp.ravel())
    ghost = np.flatnonzero(op.ghost.ravel())
    for fl in rng.choice(comp, 3, replace=False):
        up, um = u0.copy().ravel(), u0.copy().ravel()
        up[fl] += eps
        um[fl] -= eps
        fd = (L(up.reshape(g.n), beta, alpha0) - L(um.reshape(g.n), beta, alpha0)) / (2 * eps)
        assert abs(gu.ravel()[fl] - fd) <= 1e-4 * abs(fd) + 1e-10
    for fl in list(rng.choice(comp, 2, replace=False)) + list(rng.choice(ghost, 2, replace=False)):
        bp, bm = beta.copy().ravel(), beta.copy().ravel()
        bp[fl] += eps
        bm[fl] -= eps
        fd = (L(u0, bp.reshape(g.n), alpha0) - L(u0, bm.reshape(g.n), alpha0)) / (2 * eps)
        assert abs(gb.ravel()[fl] - fd) <= 1e-4 * abs(fd) + 1e-10
    fd = (L(u0, beta, alpha0 + eps) - L(u0, beta, alpha0 - eps)) / (2 * eps)
    assert abs(ga - fd) <= 1e-4 * abs(fd)
    # against the oracle's adjoint gradient
    pe = oadj.PhiEval(op, exact=False, tol=1e-12)
    Lo, gu_o, gb_o, ga_o = oadj.trajectory_gradient(op, op.from_grid(u0), dt, nsteps, alpha0, K,
                                                    op.from_grid(target), pe, nq)
    assert abs(loss.item() - Lo) <= 1e-10 * Lo
    assert np.max(np.abs(op.from_grid(gu) - gu_o)) <= 1e-10 * np.max(np.abs(gu_o))
    assert np.max(np.abs(gb.ravel() - gb_o.ravel())) <= 1e-10 * np.max(np.abs(gb_o))
    assert abs(ga - ga_o) <= 1e-10 * abs(ga_o)


def test_trajectory_gradients_mixed(lib):
    """The FP32-mixed adjoint (Krylov vectors in FP32, reductions and the
    small exponential in FP64) through the autograd wrapper: gradients with
    respect to u_0, beta and alpha against central finite differences of the
    FP64 GPU forward (1e-4 relative, up to 1e-6 of the largest entry) and
    against the oracle's FP64 gradient (1e-4 of the largest entry)."""
    from paper_2209_15095_gb300.autograd import trajectory

    g, ph, beta, op, rng = _case(n=16, seed=3)
    alpha0, K, dt, nsteps, every, nq = 1.0, 1.0, 0.02, 7, 3, 10
    ctx = _ctx(lib, g, alpha0, K, tol=1e-8, precision="mixed")
    ref_ctx = _ctx(lib, g, alpha0, K)
    dph = _dev(ph)
    u0 = op.to_grid(rng.uniform(0.2, 0.9, op.ncomp))
    target = op.to_grid(rng.uniform(0.0, 0.5, op.ncomp))
    du0 = _dev(u0).requires_grad_(True)
    dbeta = _dev(beta).requires_grad_(True)
    dalpha = torch.tensor([alpha0], dtype=torch.float64, device="cuda", requires_grad=True)
    dtarget = _dev(target)
    uT = trajectory(ctx, du0, dbeta, dalpha, dph, dt, nsteps, K=K, checkpoint_every=every, nquad=nq)
    loss = 0.5 * ((uT - dtarget) ** 2).sum()
    loss.backward()
    gu, gb, ga = du0.grad.cpu().numpy(), dbeta.grad.cpu().numpy(), dalpha.grad.item()
    gu_max, gb_max = np.max(np.abs(gu)), np.max(np.abs(gb))

    def L(u0_, beta_, alpha_):
        with torch.no_grad():
            out = trajectory(ref_ctx, _dev(u0_), _dev(beta_),
                             torch.tensor([alpha_], dtype=torch.float64, device="cuda"), dph, dt, nsteps, K=K,
                             checkpoint_every=every, nquad=nq)
            return 0.5 * float(((out - dtarget) ** 2).sum())

    eps = 1e-6
    comp = np.flatnonzero(op.comp.ravel())
    ghost = np.flatnonzero(op.ghost.ravel())
    for fl in rng.choice(comp, 3, replace=False):
        up, um = u0.copy().ravel(), u0.copy().ravel()
        up[fl] += eps
        um[fl] -= eps
        fd = (L(up.reshape(g.n), beta, alpha0) - L(um.reshape(g.n), beta, alpha0)) / (2 * eps)
        assert abs(gu.ravel()[fl] - fd) <= 1e-4 * abs(fd) + 1e-6 * gu_max, (gu.ravel()[fl], fd)
    for fl in list(rng.choice(comp, 2, replace=False)) + list(rng.choice(ghost, 2, replace=False)):
        bp, bm = beta.copy().ravel(), beta.copy().ravel()
        bp[fl] += eps
        bm[fl] -= eps
        fd = (L(u0, bp.reshape(g.n), alpha0) - L(u0, bm.reshape(g.n), alpha0)) / (2 * eps)
        assert abs(gb.ravel()[fl] - fd) <= 1e-4 * abs(fd) + 1e-6 * gb_max, (gb.ravel()[fl], fd)
    fd = (L(u0, beta, alpha0 + eps) - L(u0, beta, alpha0 - eps)) / (2 * eps)
    assert abs(ga - fd) <= 1e-4 * abs(fd), (ga, fd)
    pe = oadj.PhiEval(op, exact=False, tol=1e-12)
    Lo, gu_o, gb_o, ga_o = oadj.trajectory_gradient(op, op.from_grid(u0), dt, nsteps, alpha0, K,
                                                    op.from_grid(target), pe, nq)
    assert abs(loss.item() - Lo) <= 1e-5 * Lo
    assert np.max(np.abs(op.from_grid(gu) - gu_o)) <= 1e-4 * np.max(np.abs(gu_o))
    assert np.max(np.abs(gb.ravel() - gb_o.ravel())) <= 1e-4 * np.max(np.abs(gb_o))
    assert abs(ga - ga_o) <= 1e-4 * abs(ga_o)
