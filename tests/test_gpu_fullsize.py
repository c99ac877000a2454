"""The configured workloads at their full sizes, in the bench's launch
configuration (each workload's grid, Krylov tolerance and basis limit,
precision and step schedule), against the FP64 oracle where it computes the
result in seconds, and by properties that hold at any size where it cannot.

- Domain set-up on every workload: node kinds and the ordered point list
  bit-exact, D_p and the Gershgorin bound to 1e-12.
- One ETD step on every workload (first step: ETD1) from the workload's
  initial data: FP64 against the oracle replaying the GPU's substep and basis
  decisions (1e-10 relative), FP32-mixed against the oracle at 1e-5; the two
  species of twoball3d coupled through the competition reaction.
- One level-set step (advection, extension, Stefan speed) of star3d 128^3:
  phi within 1e-10 h (FP64; FP32-mixed 1e-6 h within 2h of the front and
  1e-4 h beyond), the extended u to 1e-10 relative.
- The explicit ETD2 step and one adjoint step of adjoint_ball3d 128^3 (beta
  field, 299k points) against the oracle (1e-10 relative).
- 20 free-boundary steps with the bench's schedule (start-up
  reinitialisation where the workload has one, reinitialisation every 5
  steps): the domain grows, 0 <= u <= 1 up to rounding, FP32-mixed within
  1e-5 of FP64 at the same Krylov tolerance, and the 4D ellipsoid's solution
  keeps its reflection symmetry in every axis.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj  # noqa: E402
from oracle import etd as oetd  # noqa: E402
from oracle import levelset  # noqa: E402
from oracle.eb import EBOperator  # noqa: E402
from oracle.grid import Grid  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    return etd


@functools.lru_cache(maxsize=None)
def _workload(name):
    from paper_2209_15095_gb300 import inputs

    return getattr(inputs, name)()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ctx(lib, w, precision, tol=None, adjoint=False):
    nsp = len(w.phi0)
    if tol is None:
        tol = w.tol if precision == "fp64" else getattr(w, "tol_mixed", w.tol)
    return lib.Context(w.n, w.lo, w.hi, nspecies=nsp, precision=precision, tol=tol, m_max=w.m_max,
                       reaction=w.reaction, rparams=w.rparams, mu=w.mu, beta=[b if np.isscalar(b) else 1.0 for b in w.beta],
                       adjoint=adjoint)


def _beta_field(w, s):
    return None if np.isscalar(w.beta[s]) else w.beta[s]


@functools.lru_cache(maxsize=None)
def _ops(name):
    """Oracle operators of the workload's species on the clamped phi_0."""
    w = _workload(name)
    g = Grid(w.n, w.lo, w.hi)
    phis = [levelset.clamp(np.asarray(p, dtype=np.float64), g.h) for p in w.phi0]
    return g, phis, [EBOperator(g, phis[s], w.beta[s]) for s in range(len(phis))]


def _prepared(lib, w, precision, name):
    """A context with the clamped phi_0 (GPU levelset_prepare without
    reinitialisation) and the domain set up, and the GPU phi fields."""
    ctx = _ctx(lib, w, precision)
    dph = [_dev(p) for p in w.phi0]
    for s in range(len(dph)):
        ctx.levelset_prepare(dph[s], False)
        bf = _beta_field(w, s)
        ctx.init_domain(s, dph[s], None if bf is None else _dev(bf))
    return ctx, dph


WORKLOADS = ["star3d", "twoball3d", "ellipsoid4d", "adjoint_ball3d"]


@pytest.mark.parametrize("name", WORKLOADS)
def test_fullsize_domain(lib, name):
    w = _workload(name)
    g, phis, ops = _ops(name)
    ctx, dph = _prepared(lib, w, "fp64", name)
    for s, op in enumerate(ops):
        # the GPU clamp is the oracle's, bit for bit
        assert np.array_equal(dph[s].cpu().numpy(), phis[s])
        dom = ctx.read_domain(s)
        ref_kind = np.where(op.comp, 2, np.where(op.ghost, 1, 0)).astype(np.uint8)
        assert np.array_equal(dom["kind"], ref_kind)
        assert dom["ncomp"] == op.ncomp
        assert np.array_equal(dom["idx"], op.index.astype(np.int32))
        assert np.max(np.abs(dom["diag"] - op.diag) / np.abs(op.diag)) < 1e-12
        assert dom["nclamp"] == op.nclamp
        assert abs(dom["gersh"] - op.gershgorin()) <= 1e-12 * op.gershgorin()


def _F(w, ops, us, s):
    """F of species s at its computational points (the other species' value
    where that point is computational for it, else 0)."""
    if w.reaction == "competition":
        o = 1 - s
        other = ops[s].from_grid(ops[o].to_grid(us[o]))
        pair = [us[s], other] if s == 0 else [other, us[s]]
        return oetd.reaction("competition", w.rparams, pair)[s]
    return oetd.reaction(w.reaction, w.rparams, [us[s]])[0]


@pytest.mark.parametrize("name,precision", [(n, p) for n in WORKLOADS for p in ("fp64", "mixed")])
def test_fullsize_etd_step(lib, name, precision):
    w = _workload(name)
    g, phis, ops = _ops(name)
    ctx, dph = _prepared(lib, w, precision, name)
    us0 = [ops[s].from_grid(np.where(ops[s].comp, w.u0[s], 0.0)) for s in range(len(ops))]
    du = [_dev(ops[s].to_grid(us0[s])) for s in range(len(ops))]
    st = ctx.step(w.dt, du, stats=True)
    tol = w.tol if precision == "fp64" else getattr(w, "tol_mixed", w.tol)
    for s, op in enumerate(ops):
        F = _F(w, ops, us0, s)  # first step: ETD1 (F_{n-1} = F_n)
        # the oracle replays the GPU's substeps and basis sizes
        forced = [(t, m, 0) for t, m in st[s]["trace"]]
        assert len(forced) == st[s]["substeps"]
        uo, _ = oetd.etd2_step(op, us0[s], F, F, w.dt, tol=tol, m_max=w.m_max, forced_trace=forced)
        ug = du[s].cpu().numpy()
        bound = 1e-10 if precision == "fp64" else 1e-5
        assert np.max(np.abs(op.from_grid(ug) - uo)) <= bound * np.max(np.abs(uo))
        assert np.all(ug[~op.comp] == 0.0)


@functools.lru_cache(maxsize=None)
def _levelset_oracle(name):
    w = _workload(name)
    g, phis, ops = _ops(name)
    u = np.where(ops[0].comp, w.u0[0], 0.0)
    ph_o, ue_o, _ = levelset.levelset_advance(phis[0], u, ops[0].comp, g, w.dt, w.mu[0], False)
    return ph_o, ue_o


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fullsize_levelset_step(lib, precision):
    name = "star3d"
    w = _workload(name)
    g, phis, ops = _ops(name)
    ctx, dph = _prepared(lib, w, precision, name)
    du = _dev(np.where(ops[0].comp, w.u0[0], 0.0))
    ctx.levelset_advance(0, dph[0], du, w.dt, False)
    ctx.sync()
    ph_o, ue_o = _levelset_oracle(name)
    ph_g = dph[0].cpu().numpy()
    assert ((ph_g < 0) == (ph_o < 0)).all()
    if precision == "fp64":
        assert np.max(np.abs(ph_g - ph_o)) <= 1e-10 * g.h
    else:
        near = np.abs(ph_o) < 2 * g.h
        assert np.max(np.abs(ph_g - ph_o)[near]) <= 1e-6 * g.h
        assert np.max(np.abs(ph_g - ph_o)) <= 1e-4 * g.h
    # FP32 extension sweeps in the mixed path: at most 11 two-pass updates of
    # at most 14 roundings each, 11 * 14 * 2^-24 = 9.2e-6 of max |u|
    bound = 1e-10 if precision == "fp64" else 1e-5
    assert np.max(np.abs(du.cpu().numpy() - ue_o)) <= bound * np.max(np.abs(ue_o))


def test_fullsize_adjoint_steps(lib):
    """adjoint_ball3d 128^3: the explicit ETD2 step and one adjoint step (beta
    field, alpha gradient, 8 Gauss-Legendre points) against the oracle."""
    w = _workload("adjoint_ball3d")
    g, phis, ops = _ops("adjoint_ball3d")
    op = ops[0]
    alpha, K = w.rparams
    ctx = lib.Context(w.n, w.lo, w.hi, nspecies=1, precision="fp64", tol=1e-12, m_max=40, reaction="logistic_ak",
                      rparams=(alpha, K), adjoint=True)
    dbeta = _dev(w.beta[0])
    ctx.init_domain(0, _dev(phis[0]), dbeta)
    rng = np.random.default_rng(5)
    u_n = op.to_grid(op.from_grid(w.u0[0]))
    u_nm1 = op.to_grid(rng.uniform(0.2, 0.9, op.ncomp))
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.step_explicit(0, w.dt, _dev(u_n), _dev(u_nm1), out, stats=True)
    pe = oadj.PhiEval(op, exact=False, tol=1e-12)
    un_c, unm1_c = op.from_grid(u_n), op.from_grid(u_nm1)
    F = oadj.reaction_ak(un_c, alpha, K)
    Fm = oadj.reaction_ak(unm1_c, alpha, K)
    # the oracle replays the GPU's Krylov decisions of the explicit step
    ref, _ = oetd.combination(op, [un_c, w.dt * F, w.dt * (F - Fm)], w.dt, tol=1e-12, m_max=40,
                              forced_trace=[(t, m, 0) for t, m in st["trace"]])
    assert np.max(np.abs(op.from_grid(out.cpu().numpy()) - ref)) <= 1e-10 * np.max(np.abs(ref))
    lam = op.to_grid(rng.standard_normal(op.ncomp))
    acc0 = op.to_grid(rng.standard_normal(op.ncomp))
    dl, da = _dev(lam), _dev(acc0)
    gb = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.adjoint_step(0, w.dt, _dev(u_n), _dev(u_nm1), False, dl, da, gb, ga, 8)
    ctx.sync()
    to_n, to_nm1, dalpha, dbeta_o = oadj.adjoint_step(op, pe, w.dt, un_c, unm1_c, op.from_grid(lam), alpha, K, 8)
    lam_ref = to_n + op.from_grid(acc0)
    # both sides evaluate every phi action to tolerance 1e-12 with their own
    # decisions: they agree to about 1e-11
    assert np.max(np.abs(op.from_grid(dl.cpu().numpy()) - lam_ref)) <= 1e-10 * np.max(np.abs(lam_ref))
    assert np.max(np.abs(op.from_grid(da.cpu().numpy()) - to_nm1)) <= 1e-10 * np.max(np.abs(to_nm1))
    assert abs(ga.item() - dalpha) <= 1e-10 * abs(dalpha)
    gbo = dbeta_o.ravel()
    assert np.max(np.abs(gb.cpu().numpy().ravel() - gbo)) <= 1e-10 * np.max(np.abs(gbo))


def _run_steps(lib, w, precision, nsteps, tol=None):
    """nsteps free-boundary steps with the bench's schedule; returns phi, u."""
    ctx = _ctx(lib, w, precision, tol=tol)
    nsp = len(w.phi0)
    dph = [_dev(p) for p in w.phi0]
    du = [_dev(np.where(w.phi0[s] < 0, w.u0[s], 0.0)) for s in range(nsp)]
    for s in range(nsp):
        ctx.levelset_prepare(dph[s], getattr(w, "reinit_at_start", False))
        ctx.init_domain(s, dph[s])
    inside0 = [int((p < 0).sum().item()) for p in dph]
    for k in range(nsteps):
        reinit = w.reinit_every > 0 and (k + 1) % w.reinit_every == 0
        for s in range(nsp):
            ctx.levelset_advance(s, dph[s], du[s], w.dt, reinit)
        for s in range(nsp):
            ctx.init_domain(s, dph[s])
        ctx.step(w.dt, du)
    ctx.sync()
    return [p.cpu().numpy() for p in dph], [u.cpu().numpy() for u in du], inside0


@pytest.mark.parametrize("name", ["star3d", "twoball3d", "ellipsoid4d"])
def test_fullsize_multistep_properties(lib, name):
    w = _workload(name)
    h = Grid(w.n, w.lo, w.hi).h
    nsteps = 20
    ph64, u64, in0 = _run_steps(lib, w, "fp64", nsteps)
    # mixed precision at the FP64 run's Krylov tolerance: the FP32 arithmetic alone
    phmx, umx, _ = _run_steps(lib, w, "mixed", nsteps, tol=w.tol)
    for s in range(len(w.phi0)):
        for ph, u in ((ph64[s], u64[s]), (phmx[s], umx[s])):
            # the Stefan speed is outward: the domain grows
            assert int((ph < 0).sum()) > in0[s]
            # logistic / competition growth from data in [0, 1] with zero
            # Dirichlet data stays in [0, 1]
            assert u.min() >= -1e-9 and u.max() <= 1.0 + 1e-9
        both = (ph64[s] < 0) & (phmx[s] < 0)
        assert np.max(np.abs(u64[s] - umx[s])[both]) <= 1e-5 * np.max(np.abs(u64[s]))
        near = np.abs(ph64[s]) < 2 * h
        assert np.max(np.abs(ph64[s] - phmx[s])[near]) <= 1e-2 * h
    if name == "ellipsoid4d":
        # the ellipsoid, its data and the grid are symmetric under x_d -> -x_d
        for d in range(4):
            for ph, u, tol in ((ph64[0], u64[0], 1e-9), (phmx[0], umx[0], 1e-5)):
                assert np.max(np.abs(u - np.flip(u, axis=d))) <= tol * np.max(np.abs(u))
                assert np.max(np.abs(ph - np.flip(ph, axis=d))) <= tol * h


def test_fullsize_star3d_mixed_operating_point(lib):
    """The mixed operating point the bench reports (star3d 128^3, Krylov
    tolerance 1.1e-6): 55 free-boundary steps with the bench's schedule (5
    warm-up and 50 timed steps), against the FP64 run at the workload's
    tolerance 1e-7: u within 1e-5 relative where both are inside, the
    interface within 1e-2 h."""
    w = _workload("star3d")
    h = Grid(w.n, w.lo, w.hi).h
    nsteps = 55
    ph64, u64, _ = _run_steps(lib, w, "fp64", nsteps)
    phmx, umx, _ = _run_steps(lib, w, "mixed", nsteps, tol=1.1e-6)
    both = (ph64[0] < 0) & (phmx[0] < 0)
    err = np.max(np.abs(u64[0] - umx[0])[both]) / np.max(np.abs(u64[0]))
    assert err <= 1e-5, err
    near = np.abs(ph64[0]) < h
    assert np.max(np.abs(ph64[0] - phmx[0])[near]) <= 1e-2 * h


def test_fullsize_ball512_mixed(lib):
    """The bandwidth stress shape the bench times (ball512: a fixed ball of
    radius 7 in a 512^3 grid, 46.3M points; the split passes on aligned
    4-node groups): two ETD2 steps in FP32-mixed against the FP64 GPU path at
    the same tolerance, within 1e-5 relative in u."""
    from paper_2209_15095_gb300 import inputs

    w = inputs.ball512()
    phi = _dev(w.phi0[0])
    u0 = _dev(w.u0[0])
    out = {}
    for precision in ("fp64", "mixed"):
        ctx = lib.Context(w.n, w.lo, w.hi, nspecies=1, precision=precision, tol=w.tol, m_max=w.m_max,
                          reaction=w.reaction, beta=w.beta)
        u = u0.clone()
        ctx.init_domain(0, phi)
        for _ in range(2):
            st = ctx.step(w.dt, [u], stats=True)
        out[precision] = u
        assert st[0]["ncomp"] > 46_000_000 and st[0]["krylov_iters"] >= 10
        del ctx
        torch.cuda.empty_cache()
    a, b = out["fp64"], out["mixed"]
    err = (torch.max(torch.abs(a - b)) / torch.max(torch.abs(a))).item()
    assert err <= 1e-5, err
