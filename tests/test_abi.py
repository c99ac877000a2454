"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/etd_gb300.h (no compute calls: no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "etd_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared()
    for required in ("etd_init_domain", "etd_step", "levelset_advance", "etd_phi_combination", "etd_create"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2209_15095_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_workspace_size_and_argument_checks():
    from paper_2209_15095_gb300 import build, etd

    lib = ctypes.CDLL(build.build())
    lib.etd_workspace_bytes.restype = ctypes.c_size_t
    g = etd.Grid()
    g.ndim = 3
    for d in range(3):
        g.n[d], g.lo[d], g.hi[d] = 32, -1.0, 1.0
    p = etd.Params()
    p.nspecies, p.precision, p.krylov_tol, p.m_max, p.reaction = 1, 0, 1e-8, 30, 1
    p.beta[0] = p.beta[1] = 1.0
    n64 = lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p))
    assert n64 > 31 * 32 ** 3 * 8  # the basis alone
    p.precision = 1
    n32 = lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p))
    assert n32 < n64
    p.m_max = 99  # out of range
    assert lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p)) == 0
    p.m_max = 30
    g.hi[1] = 2.0  # unequal spacing
    assert lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p)) == 0


def test_grid_and_parameter_bounds():
    """The size and parameter limits the header states, checked on the host
    (etd_workspace_bytes returns 0 for a rejected grid or parameter set)."""
    from paper_2209_15095_gb300 import build, etd

    lib = ctypes.CDLL(build.build())
    lib.etd_workspace_bytes.restype = ctypes.c_size_t

    def grid(ndim, n):
        g = etd.Grid()
        g.ndim = ndim
        for d in range(min(ndim, 4)):  # the struct holds 4 axes
            g.n[d], g.lo[d], g.hi[d] = n, -1.0, 1.0
        return g

    def params(**kw):
        p = etd.Params()
        p.nspecies, p.precision, p.krylov_tol, p.m_max, p.reaction = 1, 0, 1e-8, 30, 1
        p.beta[0] = p.beta[1] = 1.0
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    ok = lambda g, p: lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p)) > 0
    assert ok(grid(2, 16), params()) and ok(grid(4, 12), params())
    assert not ok(grid(1, 16), params()) and not ok(grid(5, 12), params())  # 2 <= ndim <= 4
    assert not ok(grid(3, 7), params())  # at least 8 nodes per axis
    assert not ok(grid(2, 65536), params())  # at most 65535 per axis
    assert not ok(grid(3, 1291), params())  # more than 2^31 - 1 nodes
    assert ok(grid(3, 16), params(m_max=61)) and not ok(grid(3, 16), params(m_max=62))
    assert not ok(grid(3, 16), params(m_max=4))
    for scheme in (0, 1, 2, 3, 4, 5, 6):
        assert ok(grid(3, 16), params(scheme=scheme))
    assert not ok(grid(3, 16), params(scheme=7)) and not ok(grid(3, 16), params(scheme=-1))
    # the phi_3 schemes need m_max <= 60 (the augmented matrix has m + 4 rows, at most 64)
    for scheme in (4, 5, 6):
        assert ok(grid(3, 16), params(scheme=scheme, m_max=60))
        assert not ok(grid(3, 16), params(scheme=scheme, m_max=61))
    assert not ok(grid(3, 16), params(nspecies=3)) and not ok(grid(3, 16), params(nspecies=0))
    assert not ok(grid(3, 16), params(reaction=3))  # competition needs two species
    assert ok(grid(3, 16), params(reaction=3, nspecies=2))
    assert not ok(grid(3, 16), params(krylov_tol=0.0)) and not ok(grid(3, 16), params(precision=2))
    bad_beta = params()
    bad_beta.beta[0] = 0.0
    assert not ok(grid(3, 16), bad_beta)
