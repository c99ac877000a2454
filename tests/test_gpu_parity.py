"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: node classification and the list of computational points.
1e-12 relative: row diagonals D_p and the matrix-free operator.
1e-10 relative (FP64): the phi-combination, the ETD steps, the level-set
step and whole free-boundary runs, from identical inputs, with the oracle
replaying the GPU's Krylov decisions (substep sizes and basis sizes) where
its own controller could straddle a threshold; the interface within
1e-10 h.  1e-5 relative in u (and the interface within 1e-2 h) for the
FP32-mixed path against the FP64 oracle.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etd as oetd  # noqa: E402
from oracle import krylov, levelset  # noqa: E402
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


def _shape_phi(ndim, n, box, kind):
    g = Grid((n,) * ndim, (-box,) * ndim, (box,) * ndim)
    x = g.coords()
    if kind == "ball":
        ph = np.sqrt(sum(c * c for c in x)) - 0.62 * box
    elif kind == "ellipsoid":
        a = [0.7, 0.55, 0.5, 0.45][:ndim]
        ph = np.sqrt(sum((x[d] / (a[d] * box)) ** 2 for d in range(ndim))) - 1.0
    elif kind == "peanut":
        s = box / 1.0
        X, Y = x[0] / s, x[1] / s
        ph = 0.5 - np.exp(-20 * (X ** 2 + (Y - 0.25) ** 2)) - np.exp(-20 * (X ** 2 + (Y + 0.25) ** 2))
        for d in range(2, ndim):
            ph = ph + (x[d] / s) ** 2
    return g, ph


CASES = [(2, 40, 1.0, "peanut"), (2, 33, 2.0, "ball"), (3, 20, 2.0, "ellipsoid"), (3, 24, 1.0, "peanut"),
         (4, 13, 2.0, "ball")]


def _ctx(lib, g, **kw):
    args = dict(nspecies=1, precision="fp64", tol=1e-10, m_max=40, reaction="logistic", mu=(1.0,), beta=(1.0,))
    args.update(kw)
    return lib.Context(g.n, g.lo, g.hi, **args)


@pytest.mark.parametrize("ndim,n,box,kind", CASES)
@pytest.mark.parametrize("beta_field", [False, True])
def test_domain_and_operator(lib, ndim, n, box, kind, beta_field):
    g, ph = _shape_phi(ndim, n, box, kind)
    rng = np.random.default_rng(ndim * 100 + n)
    beta = (1.0 + 0.3 * rng.uniform(-1, 1, size=g.n)) if beta_field else 1.0
    op = EBOperator(g, ph, beta)
    ctx = _ctx(lib, g)
    dph = _dev(ph)
    dbeta = _dev(beta) if beta_field else None
    ctx.init_domain(0, dph, dbeta)
    dom = ctx.read_domain(0)
    ref_kind = np.where(op.comp, 2, np.where(op.ghost, 1, 0)).astype(np.uint8)
    assert np.array_equal(dom["kind"], ref_kind)
    assert dom["ncomp"] == op.ncomp
    assert np.array_equal(dom["idx"], op.index.astype(np.int32))
    assert np.max(np.abs(dom["diag"] - op.diag) / np.abs(op.diag)) < 1e-12
    assert dom["nclamp"] == op.nclamp
    assert abs(dom["gersh"] - op.gershgorin()) <= 1e-12 * op.gershgorin()
    # y = dt C x
    dt = 0.37
    x = rng.standard_normal(g.n)
    x_c = op.from_grid(x)
    x_grid = op.to_grid(x_c)  # zero off the computational set
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ctx.apply_operator(0, dt, _dev(x_grid), y)
    yo = dt * (op.C @ x_c)
    yg = op.from_grid(y.cpu().numpy())
    assert np.max(np.abs(yg - yo)) <= 1e-12 * np.max(np.abs(yo))


def _compare_phipm(ctx, op, dt, vs, tol, m_max, stats, yg):
    apply_A = lambda x: dt * (op.C @ x)
    anorm = dt * op.gershgorin()
    yo, tr = krylov.phipm(apply_A, vs, tol, m_max, anorm)
    gtr = [(t, m) for t, m in stats["trace"]]
    if [m for _, m in gtr] != [m for _, m, _ in tr] or len(gtr) != len(tr):
        yo, tr = krylov.phipm(apply_A, vs, tol, m_max, anorm, forced_trace=[(t, m, 0) for t, m in gtr])
    return yo, tr


@pytest.mark.parametrize("ndim,n,box,kind", CASES)
def test_phi_combination_fp64(lib, ndim, n, box, kind):
    g, ph = _shape_phi(ndim, n, box, kind)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, tol=1e-10, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(7 + n)
    vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
    dt = 0.8 * g.h  # stiff enough for several substeps
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    yg = op.from_grid(y.cpu().numpy())
    yo, tr = _compare_phipm(ctx, op, dt, vs, 1e-10, 40, st, yg)
    assert np.max(np.abs(yg - yo)) <= 1e-10 * np.max(np.abs(yo)), (st, tr)
    # off the computational set the output is zero
    yfull = y.cpu().numpy()
    assert np.all(yfull[~op.comp] == 0.0)


def test_phi_combination_substeps_and_rejections(lib):
    g, ph = _shape_phi(2, 48, 2.0, "ball")
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, tol=1e-8, m_max=10)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(3)
    vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
    dt = 0.3
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    assert st["substeps"] > 3 and st["rejections"] > 0
    yg = op.from_grid(y.cpu().numpy())
    yo, _ = _compare_phipm(ctx, op, dt, vs, 1e-8, 10, st, yg)
    assert np.max(np.abs(yg - yo)) <= 1e-10 * np.max(np.abs(yo))


@pytest.mark.parametrize("ndim,n,box,kind", [(2, 40, 1.0, "peanut"), (3, 24, 2.0, "ellipsoid")])
def test_phi_combination_mixed(lib, ndim, n, box, kind):
    g, ph = _shape_phi(ndim, n, box, kind)
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, precision="mixed", tol=1e-7, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(11)
    u = rng.uniform(0, 1, op.ncomp)
    F = u * (1 - u)
    dt = g.h * g.h  # |dt C| about 4N, the stiffness of the workloads
    vs = [u, dt * F, 0.1 * dt * F]
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y)
    ctx.sync()
    yo = oetd.phi.combination_expm(dt * op.C.toarray(), vs) if op.ncomp < 3000 else None
    if yo is None:
        yo, _ = krylov.phipm(lambda x: dt * (op.C @ x), vs, 1e-12, 40, dt * op.gershgorin())
    yg = op.from_grid(y.cpu().numpy())
    assert np.max(np.abs(yg - yo)) <= 1e-5 * np.max(np.abs(yo))


@pytest.mark.parametrize("precision,n,split_min", [("fp64", 112, 1 << 17), ("mixed", 140, 1 << 18)])
def test_phi_combination_large_split_pass(lib, precision, n, split_min):
    """Problems of at least 2^17 (FP64) or 2^18 (FP32) computational points
    take the split Lanczos pass (V_j stored, then Z_j = A V_j) with several
    points in flight per thread."""
    g, ph = _shape_phi(3, n, 2.0, "ball")
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp >= split_min
    tol = 1e-10 if precision == "fp64" else 1e-7
    ctx = _ctx(lib, g, precision=precision, tol=tol, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(17)
    if precision == "fp64":
        vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
        dt = 4.0 * g.h * g.h
    else:
        u = rng.uniform(0, 1, op.ncomp)
        dt = g.h * g.h
        vs = [u, dt * u * (1 - u), 0.1 * dt * u * (1 - u)]
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    yg = op.from_grid(y.cpu().numpy())
    if precision == "fp64":
        yo, tr = _compare_phipm(ctx, op, dt, vs, tol, 40, st, yg)
        assert np.max(np.abs(yg - yo)) <= 1e-10 * np.max(np.abs(yo)), (st, tr)
    else:
        yo, _ = krylov.phipm(lambda x: dt * (op.C @ x), vs, 1e-12, 40, dt * op.gershgorin())
        assert np.max(np.abs(yg - yo)) <= 1e-5 * np.max(np.abs(yo))
    assert np.all(y.cpu().numpy()[~op.comp] == 0.0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_etd2_step_from_state(lib, precision, tol):
    g, ph = _shape_phi(3, 26, 2.0, "ellipsoid")
    beta = 1.0
    op = EBOperator(g, ph, beta)
    ctx = _ctx(lib, g, precision=precision, tol=1e-10 if precision == "fp64" else 1e-6, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(5)
    u0 = op.to_grid(rng.uniform(0, 1, op.ncomp))
    du = torch.tensor(u0, device="cuda")
    dt = 0.02
    # step 1 (ETD1: F_prev := F_0), step 2 (ETD2 with the stored F_prev)
    st1 = ctx.step(dt, [du], stats=True)
    u1g = du.cpu().numpy()
    st2 = ctx.step(dt, [du], stats=True)
    u2g = du.cpu().numpy()
    F = lambda v: v * (1 - v)
    uc0 = op.from_grid(u0)
    # FP64: the oracle at the GPU's tolerance replays its substep and basis
    # decisions; mixed: against the oracle at 1e-12
    fp64 = precision == "fp64"
    ot = 1e-10 if fp64 else 1e-12
    ft1 = forced(st1[0]["trace"]) if fp64 else None
    ft2 = forced(st2[0]["trace"]) if fp64 else None
    u1o, _ = oetd.etd2_step(op, uc0, F(uc0), F(uc0), dt, tol=ot, m_max=40, forced_trace=ft1)
    u2o, _ = oetd.etd2_step(op, u1o, F(u1o), F(uc0), dt, tol=ot, m_max=40, forced_trace=ft2)
    for ug, uo in ((u1g, u1o), (u2g, u2o)):
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= tol * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)


def test_etd2_steps_large_mixed(lib):
    """Two ETD2 steps of a large FP32-mixed problem (a ball of at least 2^18
    points, last axis a multiple of 4): the set-up (F_n, the stored F_{n-1}
    and its validity bytes, v_1, v_2), the Lanczos basis and the combination
    all run on the 4-node groups.  Step 1 is ETD1 (no F_{n-1} yet), step 2
    takes F_{n-1} from step 1; against the oracle at 1e-5."""
    g, ph = _shape_phi(3, 140, 2.0, "ball")
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp >= 1 << 18 and g.n[2] % 4 == 0
    ctx = _ctx(lib, g, precision="mixed", tol=1e-7, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(31)
    u0 = op.to_grid(rng.uniform(0, 1, op.ncomp))
    du = torch.tensor(u0, device="cuda")
    dt = 2.0 * g.h * g.h
    st1 = ctx.step(dt, [du], stats=True)
    u1g = du.cpu().numpy()
    st2 = ctx.step(dt, [du], stats=True)
    u2g = du.cpu().numpy()
    assert st1[0]["krylov_iters"] >= 5 and st2[0]["krylov_iters"] >= 5
    F = lambda v: v * (1 - v)
    uc0 = op.from_grid(u0)
    u1o, _ = oetd.etd2_step(op, uc0, F(uc0), F(uc0), dt, tol=1e-12, m_max=40)
    u2o, _ = oetd.etd2_step(op, u1o, F(u1o), F(uc0), dt, tol=1e-12, m_max=40)
    for ug, uo in ((u1g, u1o), (u2g, u2o)):
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= 1e-5 * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)
    # the ETD2 correction itself (the F_{n-1} term) is resolved: step 2 from
    # the ETD1 form would differ by more than the bound
    u2e, _ = oetd.etd2_step(op, u1o, F(u1o), F(u1o), dt, tol=1e-12, m_max=40)
    assert np.max(np.abs(u2e - u2o)) > 10 * 1e-5 * np.max(np.abs(u2o))


@pytest.mark.parametrize("scheme", ["etd1", "etd2rk"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_etd1_etd2rk_steps_from_state(lib, scheme, precision, tol):
    """Two steps of ETD1 or ETD2RK (Sec. 3.1-3.2) through etd_step against the
    oracle; ETD2RK runs two Krylov evaluations per step and the statistics
    add both."""
    g, ph = _shape_phi(3, 26, 2.0, "ellipsoid")
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, precision=precision, tol=1e-10 if precision == "fp64" else 1e-6, m_max=40, scheme=scheme)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(9)
    u0 = op.to_grid(rng.uniform(0, 1, op.ncomp))
    du = torch.tensor(u0, device="cuda")
    dt = 0.02
    F = lambda v: v * (1 - v)
    uo = op.from_grid(u0)
    fp64 = precision == "fp64"
    ot = 1e-10 if fp64 else 1e-12
    for _ in range(2):
        st = ctx.step(dt, [du], stats=True)[0]
        ug = du.cpu().numpy()
        if scheme == "etd1":
            ft = forced(st["trace"]) if fp64 else None
            uo, _ = oetd.etd1_step(op, uo, F(uo), dt, tol=ot, m_max=40, forced_trace=ft)
        else:
            assert st["substeps"] >= 2 and len(st["trace"]) == st["substeps"]
            fts = split_evaluations(st["trace"], 2) if fp64 else None
            uo, _, _ = oetd.etd2rk_step(op, uo, lambda v, t: F(v), 0.0, dt, tol=ot, m_max=40, forced_traces=fts)
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= tol * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)


def test_levelset_step_matches(lib):
    from paper_2209_15095_gb300 import inputs

    w = inputs.disc2d()
    g = Grid(w.n, w.lo, w.hi)
    ph = levelset.clamp(w.phi0[0], g.h)
    op = EBOperator(g, ph, 1.0)
    u = np.where(op.comp, w.u0[0], 0.0)
    ctx = _ctx(lib, g, tol=w.tol, m_max=w.m_max, mu=w.mu)
    dph = _dev(ph)
    du = _dev(u)
    ctx.init_domain(0, dph)
    for reinit in (False, True):
        ph_o, ue_o, _ = levelset.levelset_advance(ph, u, op.comp, g, w.dt, w.mu[0], reinit)
        dph2, du2 = dph.clone(), du.clone()
        ctx.levelset_advance(0, dph2, du2, w.dt, reinit)
        ctx.sync()
        assert np.max(np.abs(dph2.cpu().numpy() - ph_o)) <= 1e-10 * g.h
        assert np.max(np.abs(du2.cpu().numpy() - ue_o)) <= 1e-10 * np.max(np.abs(ue_o))


@pytest.mark.parametrize("ndim", [3, 4])
def test_levelset_step_matches_nd(lib, ndim):
    n = {3: 28, 4: 22}[ndim]
    g, ph0 = _shape_phi(ndim, n, 3.0, "ellipsoid")
    ph = levelset.clamp(ph0, g.h)
    if ndim == 3:
        ph = levelset.reinit(ph, g.h)
    op = EBOperator(g, ph, 1.0)
    x = g.coords()
    r = np.sqrt(sum(c * c for c in x))
    u = np.where(op.comp, np.cos(0.3 * r), 0.0)
    ctx = _ctx(lib, g, mu=(1.3,))
    dph, du = _dev(ph), _dev(u)
    ctx.init_domain(0, dph)
    reinit = ndim == 3
    ph_o, ue_o, _ = levelset.levelset_advance(ph, u, op.comp, g, 0.02, 1.3, reinit)
    ctx.levelset_advance(0, dph, du, 0.02, reinit)
    ctx.sync()
    assert np.max(np.abs(dph.cpu().numpy() - ph_o)) <= 1e-10 * g.h
    assert np.max(np.abs(du.cpu().numpy() - ue_o)) <= 1e-10 * np.max(np.abs(ue_o))


@pytest.mark.parametrize("kind", ["plane", "ellipsoid"])
def test_reinit_fine_spacing(lib, kind):
    """Reinitialisation (Sec. 4.3) on a 3D grid with h ~ 1e-4.  On flat data
    the WENO5 weight sums W are ~10 eps'^4 with eps' = 4e-6 h^2, so their
    products per axis fall below 2^-333 and the kernel divides once per axis
    instead of once per node (the plane, |grad phi| = 1.3, is flat wherever it
    is not clamped); the ellipsoid's curved stencils keep the one shared
    division.  Both must match the oracle at 1e-10 h."""
    n, box = 24, 1.2e-3
    g = Grid((n,) * 3, (-box,) * 3, (box,) * 3)
    x = g.coords()
    if kind == "plane":
        nv = np.array([0.48, 0.6, 0.64])
        nv /= np.linalg.norm(nv)
        ph0 = 1.3 * (nv[0] * x[0] + nv[1] * x[1] + nv[2] * x[2] - 0.1 * box)
    else:
        a = (0.7, 0.55, 0.5)
        ph0 = box * (np.sqrt(sum((x[d] / (a[d] * box)) ** 2 for d in range(3))) - 1.0)
    ph = levelset.clamp(ph0, g.h)
    ref = levelset.reinit(ph, g.h)
    assert np.max(np.abs(ref - ph)) > 1e-3 * g.h  # the reinitialisation moves phi
    ctx = _ctx(lib, g)
    dph = _dev(ph)
    ctx.levelset_prepare(dph, True)
    ctx.sync()
    assert np.max(np.abs(dph.cpu().numpy() - ref)) <= 1e-10 * g.h


def test_free_boundary_disc_multistep(lib):
    from oracle.freeboundary import FreeBoundary, Species
    from paper_2209_15095_gb300 import inputs

    w = inputs.disc2d()
    g = Grid(w.n, w.lo, w.hi)
    fb = FreeBoundary(g, [Species(w.phi0[0], w.u0[0], 1.0, w.mu[0])], w.reaction, w.rparams, w.tol, w.m_max,
                      reinit_every=w.reinit_every)
    ctx = _ctx(lib, g, tol=w.tol, m_max=w.m_max, mu=w.mu)
    dph = _dev(w.phi0[0])
    du = _dev(np.where(w.phi0[0] < 0, w.u0[0], 0.0))
    ctx.levelset_prepare(dph, False)
    ctx.init_domain(0, dph)
    nsteps = 12
    for k in range(nsteps):
        ctx.levelset_advance(0, dph, du, w.dt, (k + 1) % w.reinit_every == 0)
        ctx.init_domain(0, dph)
        st = ctx.step(w.dt, [du], stats=True)
        # the oracle replays the GPU's Krylov decisions of the step
        fb.step(w.dt, forced_traces=[forced(st[0]["trace"])])
    ctx.sync()
    ph_g, u_g = dph.cpu().numpy(), du.cpu().numpy()
    ph_o, u_o = fb.sp[0].phi, fb.sp[0].u
    both = (ph_g < 0) == (ph_o < 0)
    assert both.all()
    assert np.max(np.abs(ph_g - ph_o)) <= 1e-10 * g.h
    assert np.max(np.abs(u_g - u_o)) <= 1e-10 * np.max(np.abs(u_o))
    # nodes that entered the domain during the run (their F_{n-1} starts as
    # F_n, the reading for points that were not computational): same values
    entered = (ph_o < -1e-12) & (w.phi0[0] >= 0)
    assert entered.sum() > 0
    assert np.max(np.abs(u_g - u_o)[entered]) <= 1e-10 * np.max(np.abs(u_o))


def test_two_species_competition_multistep(lib):
    """Row a9: two species with their own level sets, coupled through the
    competition reaction, several free-boundary steps against the oracle."""
    from oracle.freeboundary import FreeBoundary, Species

    n = 36
    g = Grid((n,) * 3, (-3.0,) * 3, (3.0,) * 3)
    x, y, z = g.coords()
    phis, us = [], []
    for cx in (-1.0, 1.0):
        r = np.sqrt((x - cx) ** 2 + y * y + z * z)
        phis.append(r - 0.9)
        us.append(np.where(r < 0.9, np.cos(np.pi * r / 1.8), 0.0))
    beta, mu, rp = (1.0, 0.5), (1.0, 0.8), (0.5, 0.8, 1.2)
    dt, tol, m_max, nsteps = 5e-3, 1e-8, 30, 6
    fb = FreeBoundary(g, [Species(phis[s], us[s], beta[s], mu[s]) for s in range(2)], "competition", rp, tol, m_max,
                      reinit_every=5)
    ctx = lib.Context(g.n, g.lo, g.hi, nspecies=2, precision="fp64", tol=tol, m_max=m_max, reaction="competition",
                      rparams=rp, mu=mu, beta=beta)
    dph = [_dev(p) for p in phis]
    du = [_dev(np.where(phis[s] < 0, us[s], 0.0)) for s in range(2)]
    for s in range(2):
        ctx.levelset_prepare(dph[s], False)
        ctx.init_domain(s, dph[s])
    for k in range(nsteps):
        for s in range(2):
            ctx.levelset_advance(s, dph[s], du[s], dt, (k + 1) % 5 == 0)
        for s in range(2):
            ctx.init_domain(s, dph[s])
        st = ctx.step(dt, du, stats=True)
        fb.step(dt, forced_traces=[forced(st[s]["trace"]) for s in range(2)])
    ctx.sync()
    for s in range(2):
        ph_g, u_g = dph[s].cpu().numpy(), du[s].cpu().numpy()
        ph_o, u_o = fb.sp[s].phi, fb.sp[s].u
        assert ((ph_g < 0) == (ph_o < 0)).all()
        assert np.max(np.abs(ph_g - ph_o)) <= 1e-10 * g.h
        assert np.max(np.abs(u_g - u_o)) <= 1e-10 * np.max(np.abs(u_o))


def test_levelset_step_mixed_precision(lib):
    """FP32-mixed path: WENO5/Godunov arithmetic in FP32 except the
    reinitialisation within h of the interface, extension sweeps in FP32;
    against the FP64 oracle.  Bound on the extended u: each FP32 two-pass
    sweep update is a convex combination of at most 1 + N + N^2 = 13 terms,
    rounded at most 14 times (unit roundoff 2^-24), and the passes do not
    expand errors, so ceil(21 / 2) = 11 updates stay within
    11 * 14 * 2^-24 = 9.2e-6 of max |u|."""
    g, ph0 = _shape_phi(3, 28, 3.0, "ellipsoid")
    ph = levelset.reinit(levelset.clamp(ph0, g.h), g.h)
    op = EBOperator(g, ph, 1.0)
    x = g.coords()
    r = np.sqrt(sum(c * c for c in x))
    u = np.where(op.comp, np.cos(0.3 * r), 0.0)
    ctx = _ctx(lib, g, precision="mixed", tol=1e-6, mu=(1.3,))
    dph, du = _dev(ph), _dev(u)
    ctx.init_domain(0, dph)
    ph_o, ue_o, _ = levelset.levelset_advance(ph, u, op.comp, g, 0.02, 1.3, True)
    ctx.levelset_advance(0, dph, du, 0.02, True)
    ctx.sync()
    ph_g = dph.cpu().numpy()
    near = np.abs(ph_o) < 2 * g.h
    assert ((ph_g < 0) == (ph_o < 0)).all()
    assert np.max(np.abs(ph_g - ph_o)[near]) <= 1e-6 * g.h
    assert np.max(np.abs(ph_g - ph_o)) <= 1e-4 * g.h
    assert np.max(np.abs(du.cpu().numpy() - ue_o)) <= 1e-5 * np.max(np.abs(ue_o))
    # off the swept region u is the FP64 input, untouched
    off = (np.abs(ue_o - u) == 0) & op.comp
    assert np.array_equal(du.cpu().numpy()[off], u[off])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_star_free_boundary_at_matched_tolerance(lib, precision):
    """The star-shaped 3D workload (48^3 on [-3, 3]^3) over 10 free-boundary
    steps with two reinitialisations, GPU against the FP64 oracle at the same
    Krylov tolerance.  Mixed precision stays within 1e-5 relative in u and
    1e-2 h at the interface; its FP32 arithmetic contributes far less than a
    looser Krylov tolerance would (on star3d, tolerance 1e-5 moves u by about
    1.6e-5 in FP64 and in mixed precision alike)."""
    from oracle.freeboundary import FreeBoundary, Species
    from paper_2209_15095_gb300 import inputs

    w = inputs.star3d(n=48, box=3.0)
    g = Grid(w.n, w.lo, w.hi)
    fb = FreeBoundary(g, [Species(w.phi0[0], w.u0[0], 1.0, w.mu[0])], w.reaction, w.rparams, w.tol, w.m_max,
                      reinit_every=w.reinit_every, reinit_at_start=True)
    ctx = _ctx(lib, g, precision=precision, tol=w.tol, m_max=w.m_max, mu=w.mu)
    dph = _dev(w.phi0[0])
    du = _dev(np.where(w.phi0[0] < 0, w.u0[0], 0.0))
    ctx.levelset_prepare(dph, True)
    ctx.init_domain(0, dph)
    for k in range(10):
        ctx.levelset_advance(0, dph, du, w.dt, (k + 1) % w.reinit_every == 0)
        ctx.init_domain(0, dph)
        st = ctx.step(w.dt, [du], stats=True)
        # FP64: the oracle replays the GPU's Krylov decisions; mixed: its own
        fb.step(w.dt, forced_traces=[forced(st[0]["trace"])] if precision == "fp64" else None)
    ctx.sync()
    ph_g, u_g = dph.cpu().numpy(), du.cpu().numpy()
    ph_o, u_o = fb.sp[0].phi, fb.sp[0].u
    assert ((ph_g < 0) == (ph_o < 0)).all()
    near = np.abs(ph_o) < g.h
    if precision == "fp64":
        assert np.max(np.abs(ph_g - ph_o)) <= 1e-10 * g.h
        assert np.max(np.abs(u_g - u_o)) <= 1e-10 * np.max(np.abs(u_o))
    else:
        assert np.max(np.abs(ph_g - ph_o)[near]) <= 1e-2 * g.h
        assert np.max(np.abs(u_g - u_o)) <= 1e-5 * np.max(np.abs(u_o))


@pytest.mark.parametrize("ndim,n", [(2, 944), (3, 139), (4, 56)])
def test_phi_combination_mixed_large_layouts(lib, ndim, n):
    """Large FP32 problems (at least 2^18 points): with the last axis a
    multiple of 4 nodes (944, 56) the split Lanczos passes run on aligned
    groups of 4 nodes; with 139 they keep the per-point loop.  Both against
    the FP64 oracle at 1e-5, one and two calls on the same context."""
    g = Grid((n,) * ndim, (-2.0,) * ndim, (2.0,) * ndim)
    ph = np.sqrt(sum(c * c for c in g.coords())) - 1.24
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp >= 1 << 18
    ctx = _ctx(lib, g, precision="mixed", tol=1e-7, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(23)
    u = rng.uniform(0, 1, op.ncomp)
    dt = g.h * g.h
    vs = [u, dt * u * (1 - u), 0.1 * dt * u * (1 - u)]
    yo, _ = krylov.phipm(lambda x: dt * (op.C @ x), vs, 1e-12, 40, dt * op.gershgorin())
    for _ in range(2):
        y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
        assert st["krylov_iters"] >= 5
        yg = op.from_grid(y.cpu().numpy())
        assert np.max(np.abs(yg - yo)) <= 1e-5 * np.max(np.abs(yo))
        assert np.all(y.cpu().numpy()[~op.comp] == 0.0)


@pytest.mark.parametrize("shape", [(144, 144, 144), (131, 123, 176)])
def test_phi_combination_mixed_3d_ragged(lib, shape):
    """Large 3D FP32 problems (at least 2^18 points, the split passes on
    aligned 4-node groups) on a cube and on a grid with unequal axes, an
    ellipsoid close to the box on every axis.  Against the FP64 oracle at
    1e-5, two calls on the same context."""
    box = 2.0
    h = 2 * box / (shape[2] - 1)
    lo = tuple(-0.5 * h * (n - 1) for n in shape)
    g = Grid(shape, lo, tuple(-v for v in lo))
    x = g.coords()
    semi = (0.43 * h * shape[0], 0.45 * h * shape[1], 0.40 * h * shape[2])
    ph = np.sqrt(sum((x[d] / semi[d]) ** 2 for d in range(3))) - 1.0
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp >= 1 << 18
    ctx = _ctx(lib, g, precision="mixed", tol=1e-7, m_max=40)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(29)
    u = rng.uniform(0, 1, op.ncomp)
    dt = g.h * g.h
    vs = [u, dt * u * (1 - u), 0.1 * dt * u * (1 - u)]
    yo, _ = krylov.phipm(lambda v: dt * (op.C @ v), vs, 1e-12, 40, dt * op.gershgorin())
    for call in range(2):
        y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
        assert st["krylov_iters"] >= 10
        yg = op.from_grid(y.cpu().numpy())
        err = np.abs(yg - yo)
        bad = np.flatnonzero(err > 1e-5 * np.max(np.abs(yo)))
        where = [tuple(int(i) for i in np.unravel_index(int(op.index[b]), g.n)) for b in bad[:8]]
        assert bad.size == 0, (call, bad.size, float(err.max()), where, st)
        assert np.all(y.cpu().numpy()[~op.comp] == 0.0)
