"""etd_phi_combination_noalloc, the entry point for callers that may not
allocate device memory (a host whose own allocator owns the whole GPU, or a
deployment that forbids allocation while running), must give the same
result as the context path (etd_init_domain + etd_phi_combination), call
after call, although every call reuses one fixed device array.

Collected last on purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _grid_struct(etd, n, lo, hi):
    g = etd.Grid()
    g.ndim = len(n)
    for d in range(len(n)):
        g.n[d], g.lo[d], g.hi[d] = n[d], lo[d], hi[d]
    return g


def _case(ndim, n, box, seed):
    lo, hi = (-box,) * ndim, (box,) * ndim
    axes = [np.linspace(-box, box, n) for _ in range(ndim)]
    xs = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(c * c for c in xs))
    if ndim == 2:
        X, Y = xs[0] / box, xs[1] / box
        phi = 0.5 - np.exp(-20 * (X ** 2 + (Y - 0.25) ** 2)) - np.exp(-20 * (X ** 2 + (Y + 0.25) ** 2))
    else:
        phi = r - 0.6 * box
    rng = np.random.default_rng(seed)
    vs = [np.where(phi < 0, rng.standard_normal(phi.shape), 0.0) for _ in range(3)]
    return (n,) * ndim, lo, hi, phi, vs


def test_noalloc_matches_context_path_twice():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    lib = etd.library()
    f = lib.etd_phi_combination_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(etd.Grid), ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                  ctypes.c_void_p]
    stream = torch.cuda.current_stream()
    # two calls in a row on different problems: nothing of the first may leak
    for ndim, n, box, seed, beta, dt in ((3, 24, 2.0, 1, 1.0, 0.05), (2, 64, 1.0, 2, 0.7, 2e-3)):
        shape, lo, hi, phi, vs = _case(ndim, n, box, seed)
        dphi = torch.tensor(phi, dtype=torch.float64, device="cuda")
        dv = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in vs]
        # context path
        ctx = etd.Context(shape, lo, hi, nspecies=1, precision="fp64", tol=1e-10, m_max=30, reaction="none",
                          beta=(beta,))
        y_ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
        ctx.init_domain(0, dphi)
        ctx.phi_combination(0, dt, dv[0], dv[1], dv[2], y_ref)
        ctx.sync()
        # fixed-array path
        y = torch.full(shape, 7.0, dtype=torch.float64, device="cuda")
        g = _grid_struct(etd, shape, lo, hi)
        rc = f(ctypes.byref(g), dphi.data_ptr(), beta, dt, dv[0].data_ptr(), dv[1].data_ptr(), dv[2].data_ptr(),
               y.data_ptr(), 1e-10, 30, stream.cuda_stream)
        assert rc == 0
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))
        assert np.all(a[b == 0.0] == 0.0)
    # the largest documented problem: 32768 nodes (32^3) with m_max = 30
    shape, lo, hi, phi, vs = _case(3, 32, 2.0, 3)
    dphi = torch.tensor(phi, dtype=torch.float64, device="cuda")
    dv = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in vs]
    ctx = etd.Context(shape, lo, hi, nspecies=1, precision="fp64", tol=1e-10, m_max=30, reaction="none",
                      beta=(1.0,))
    y_ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
    ctx.init_domain(0, dphi)
    ctx.phi_combination(0, 0.05, dv[0], dv[1], dv[2], y_ref)
    ctx.sync()
    y = torch.full(shape, 7.0, dtype=torch.float64, device="cuda")
    g = _grid_struct(etd, shape, lo, hi)
    rc = f(ctypes.byref(g), dphi.data_ptr(), 1.0, 0.05, dv[0].data_ptr(), dv[1].data_ptr(), dv[2].data_ptr(),
           y.data_ptr(), 1e-10, 30, stream.cuda_stream)
    assert rc == 0
    a, b = y.cpu().numpy(), y_ref.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))
    assert np.all(a[b == 0.0] == 0.0)
    # sizes beyond the fixed array are refused before any launch
    big = _grid_struct(etd, (40, 40, 40), (-1.0,) * 3, (1.0,) * 3)
    rc = f(ctypes.byref(big), dphi.data_ptr(), 1.0, 0.01, dv[0].data_ptr(), dv[1].data_ptr(), dv[2].data_ptr(),
           y.data_ptr(), 1e-8, 30, stream.cuda_stream)
    assert rc == -3  # ETD_ERR_WORKSPACE
    g = _grid_struct(etd, (24, 24, 24), (-2.0,) * 3, (2.0,) * 3)
    rc = f(ctypes.byref(g), dphi.data_ptr(), 1.0, 0.01, dv[0].data_ptr(), dv[1].data_ptr(), dv[2].data_ptr(),
           y.data_ptr(), 1e-8, 31, stream.cuda_stream)
    assert rc == -3
