"""Edge cases of the GPU path through the C ABI, against the FP64 oracle:
an empty domain (no node inside), a domain whose inside nodes are all ghosts,
a domain of 8 computational points (Krylov happy breakdown below 5 vectors),
the largest Krylov basis (m_max = 61: an augmented matrix of 64 rows, with
rejections at m_max), a domain reaching into the box margin (ETD_ERR_DOMAIN)
a non-finite field (ETD_ERR_NONFINITE), a device wait that reaches its
limit (ETD_ERR_TIMEOUT) and a tolerance no substep can meet
(ETD_ERR_KRYLOV): errors are reported, nothing hangs.  Grids whose rows are whole 32-node words (the word-parallel
classification), down to one word per row, in 2D-4D, with their margin
error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etd as oetd  # noqa: E402
from oracle import krylov, levelset  # noqa: E402
from oracle.eb import EBOperator  # noqa: E402
from oracle.grid import Grid  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    return etd


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ctx(lib, g, **kw):
    args = dict(nspecies=1, precision="fp64", tol=1e-10, m_max=40, reaction="logistic", mu=(1.0,), beta=(1.0,))
    args.update(kw)
    return lib.Context(g.n, g.lo, g.hi, **args)


@pytest.mark.parametrize("R_over_h", [0.0, 1.5])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_no_computational_point(lib, R_over_h, precision):
    """No node inside (R = 0: phi > 0 everywhere), or inside nodes that are
    all ghosts (R = 1.5 h): no computational point.  The step leaves u = 0
    everywhere, the combination gives 0, and the level-set step matches the
    oracle (the Stefan speed is 0)."""
    g = Grid((24, 24, 24), (-2.0,) * 3, (2.0,) * 3)
    ph = levelset.clamp(g.radius() - R_over_h * g.h + (0.3 if R_over_h == 0 else 0.0), g.h)
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp == 0 and (R_over_h == 0 or op.ghost.any())
    ctx = _ctx(lib, g, precision=precision)
    dph = _dev(ph)
    ctx.init_domain(0, dph)
    dom = ctx.read_domain(0)
    assert dom["ncomp"] == 0 and np.array_equal(dom["kind"], np.where(op.ghost, 1, 0).astype(np.uint8))
    u = torch.full(g.n, 0.3, dtype=torch.float64, device="cuda")
    st = ctx.step(0.01, [u], stats=True)[0]
    assert st["ncomp"] == 0 and torch.count_nonzero(u).item() == 0
    y = torch.full(g.n, 7.0, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(y)
    ctx.phi_combination(0, 0.01, z + 1.0, z + 1.0, z + 1.0, y)
    ctx.sync()
    assert torch.count_nonzero(y).item() == 0
    uu = torch.zeros_like(y)
    ctx.levelset_advance(0, dph, uu, 0.01, False)
    ctx.sync()
    ph_o, ue_o, _ = levelset.levelset_advance(ph, np.zeros(g.n), op.comp, g, 0.01, 1.0, False)
    assert np.max(np.abs(dph.cpu().numpy() - ph_o)) <= 1e-12 * g.h
    assert np.max(np.abs(uu.cpu().numpy())) == 0.0 and np.max(np.abs(ue_o)) == 0.0


def test_eight_point_domain(lib):
    """A ball of radius 1.75 h: 8 computational points; the Krylov basis
    breaks down (happy breakdown) before the first check at 5 vectors."""
    g = Grid((16, 16, 16), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.75 * g.h
    op = EBOperator(g, ph, 1.0)
    assert op.ncomp == 8
    ctx = _ctx(lib, g, tol=1e-12)
    ctx.init_domain(0, _dev(ph))
    dom = ctx.read_domain(0)
    assert np.array_equal(dom["idx"], op.index.astype(np.int32))
    assert np.max(np.abs(dom["diag"] - op.diag) / np.abs(op.diag)) < 1e-12
    rng = np.random.default_rng(4)
    u0 = rng.uniform(0.2, 0.8, 8)
    du = _dev(op.to_grid(u0))
    dt = 0.05
    st = ctx.step(dt, [du], stats=True)[0]
    assert max(m for _, m in st["trace"]) <= 8
    F = u0 * (1 - u0)
    uo = oetd.etd2_step(op, u0, F, F, dt, exact=True)[0]
    assert np.max(np.abs(op.from_grid(du.cpu().numpy()) - uo)) <= 1e-10 * np.max(np.abs(uo))


def test_largest_basis(lib):
    """m_max = 61 (augmented matrix of 61 + 2 + 1 = 64 rows: both halves of
    the warp's small exponential), reached with rejections: against the
    oracle replaying the GPU's decisions."""
    g = Grid((40, 40, 40), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.5
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g, tol=1e-12, m_max=61)
    ctx.init_domain(0, _dev(ph))
    rng = np.random.default_rng(3)
    vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
    dt = 0.5
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = ctx.phi_combination(0, dt, *[_dev(op.to_grid(v)) for v in vs], y, stats=True)
    assert max(m for _, m in st["trace"]) == 61 and st["rejections"] > 0
    yo, _ = krylov.phipm(lambda x: dt * (op.C @ x), vs, 1e-12, 61, dt * op.gershgorin(),
                         forced_trace=[(t, m, 0) for t, m in st["trace"]])
    assert np.max(np.abs(op.from_grid(y.cpu().numpy()) - yo)) <= 1e-10 * np.max(np.abs(yo))


def test_domain_in_box_margin_is_reported(lib):
    """An inside node within 3 nodes of the box edge: ETD_ERR_DOMAIN at the
    next synchronising call (the kernels keep every access in bounds)."""
    g = Grid((24, 24, 24), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.9
    ctx = _ctx(lib, g)
    ctx.init_domain(0, _dev(ph))
    with pytest.raises(lib.EtdError) as e:
        ctx.sync()
    assert e.value.name == "ETD_ERR_DOMAIN"


def test_nonfinite_field_is_reported(lib):
    """A NaN in u at a computational point: ETD_ERR_NONFINITE, and the
    kernel returns (every CTA takes the same decision from the same sums)."""
    g = Grid((24, 24, 24), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.2
    op = EBOperator(g, ph, 1.0)
    ctx = _ctx(lib, g)
    ctx.init_domain(0, _dev(ph))
    u = op.to_grid(np.full(op.ncomp, 0.5))
    u.ravel()[op.index[op.ncomp // 2]] = np.nan
    du = _dev(u)
    with pytest.raises(lib.EtdError) as e:
        ctx.step(0.01, [du], stats=True)
    assert e.value.name == "ETD_ERR_NONFINITE"


def _aniso(shape, h=0.1):
    """A grid of the given shape and spacing h, centred on the origin."""
    half = [0.5 * h * (n - 1) for n in shape]
    return Grid(tuple(shape), tuple(-x for x in half), tuple(half))


@pytest.mark.parametrize("shape", [(40, 32), (24, 64), (20, 18, 32), (14, 16, 96), (14, 14, 14, 32)])
def test_word_rows_domain(lib, shape):
    """Rows of whole 32-node words take the word-parallel classification
    (one word per row when the last axis is 32: both box edges in one word).
    An ellipsoid 3.5 h from every edge and a random-sign interior: kinds,
    indices, D_p and the Gershgorin bound against the oracle, bit-exact
    where integer."""
    g = _aniso(shape)
    x = g.coords()
    semi = [0.5 * g.h * (n - 1) - 3.5 * g.h for n in shape]
    ph_ball = np.sqrt(sum((x[d] / semi[d]) ** 2 for d in range(len(shape)))) - 1.0
    rng = np.random.default_rng(sum(shape))
    ph_rand = np.ones(g.n)
    inner = tuple(slice(4, n - 4) for n in shape)
    ph_rand[inner] = rng.uniform(-1.0, 0.3, size=ph_rand[inner].shape)
    for ph, full in ((ph_ball, True), (ph_rand, False)):
        op = EBOperator(g, ph, 1.0)
        ctx = _ctx(lib, g)
        ctx.init_domain(0, _dev(ph))
        dom = ctx.read_domain(0)
        ref_kind = np.where(op.comp, 2, np.where(op.ghost, 1, 0)).astype(np.uint8)
        assert np.array_equal(dom["kind"], ref_kind)
        assert dom["ncomp"] == op.ncomp
        assert np.array_equal(dom["idx"], op.index.astype(np.int32))
        if full:
            assert np.max(np.abs(dom["diag"] - op.diag) / np.abs(op.diag)) < 1e-12
            assert abs(dom["gersh"] - op.gershgorin()) <= 1e-12 * op.gershgorin()


@pytest.mark.parametrize("shape", [(32, 32, 32), (40, 64)])
def test_word_rows_margin_is_reported(lib, shape):
    """The word-parallel classification reports an inside node within 3
    nodes of the box edge (ETD_ERR_DOMAIN), as the per-node one does."""
    g = _aniso(shape)
    x = g.coords()
    # a ball touching the last axis' edge region: inside nodes at index 2
    ph = np.sqrt(sum(c * c for c in x[:-1]) + (x[-1] - x[-1].max() + 2.5 * g.h) ** 2) - 0.45
    assert (ph < 0)[..., -3].any()
    ctx = _ctx(lib, g)
    ctx.init_domain(0, _dev(ph))
    with pytest.raises(lib.EtdError) as e:
        ctx.sync()
    assert e.value.name == "ETD_ERR_DOMAIN"


def test_device_wait_timeout_is_reported(lib):
    """A device wait that reaches its limit: with a 1 ns limit on the grid
    barriers, some barrier of the phi-combination gives up, every CTA
    returns, and ETD_ERR_TIMEOUT is reported at the next synchronising call.
    With the default limit restored, the same context gives the result of a
    fresh context bit for bit.  No wait is unbounded, so nothing can hang."""
    g = Grid((64, 64, 64), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.3
    op = EBOperator(g, ph, 1.0)
    rng = np.random.default_rng(41)
    vs = [_dev(op.to_grid(rng.standard_normal(op.ncomp))) for _ in range(3)]
    ctx = _ctx(lib, g, tol=1e-10)
    ctx.init_domain(0, _dev(ph))
    ctx.sync()
    ctx.set_wait_limit(1e-9)
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    names = []
    for _ in range(5):
        try:
            ctx.phi_combination(0, 0.05, *vs, y)
            ctx.sync()
            names.append("ok")
        except lib.EtdError as e:
            names.append(e.name)
            break
    assert names[-1] == "ETD_ERR_TIMEOUT", names
    ctx.set_wait_limit(0)
    ctx.phi_combination(0, 0.05, *vs, y)
    ctx.sync()
    ref = _ctx(lib, g, tol=1e-10)
    ref.init_domain(0, _dev(ph))
    y_ref = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ref.phi_combination(0, 0.05, *vs, y_ref)
    ref.sync()
    assert torch.equal(y, y_ref)


def test_krylov_failure_is_reported(lib):
    """A tolerance that no substep can meet (1e-300 with m_max = 5 on a
    problem far larger than the basis): the controller shrinks tau below
    tau_min = 1e-6 and reports ETD_ERR_KRYLOV; the context stays usable."""
    g = Grid((32, 32, 32), (-2.0,) * 3, (2.0,) * 3)
    ph = g.radius() - 1.4
    op = EBOperator(g, ph, 1.0)
    rng = np.random.default_rng(43)
    vs = [_dev(op.to_grid(rng.standard_normal(op.ncomp))) for _ in range(3)]
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    for precision in ("fp64", "mixed"):
        ctx = _ctx(lib, g, tol=1e-300, m_max=5, precision=precision)
        ctx.init_domain(0, _dev(ph))
        with pytest.raises(lib.EtdError) as e:
            ctx.phi_combination(0, 0.5, *vs, y, stats=True)
        assert e.value.name == "ETD_ERR_KRYLOV"
        # the domain is still set up and the context answers
        assert ctx.read_domain(0, arrays=False)["ncomp"] == op.ncomp
