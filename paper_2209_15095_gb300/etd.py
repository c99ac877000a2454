"""Thin ctypes binding over the C ABI in include/etd_gb300.h.

Argument marshalling only: tensors are checked (CUDA, float64, contiguous,
full grid) and their device pointers passed through; every step of the
method runs in the library's kernels.  There is no fallback: importing this
module raises if the library is missing or no CUDA device is present.
PyTorch provides the device memory (the workspace and the fields) and the
stream (the current torch stream at context creation).
"""
import ctypes
import os

import torch

from . import build as _build

ETD_OK = 0
_ERRORS = {
    -1: "ETD_ERR_ARG",
    -2: "ETD_ERR_CUDA",
    -3: "ETD_ERR_WORKSPACE",
    -4: "ETD_ERR_KRYLOV",
    -5: "ETD_ERR_DOMAIN",
    -6: "ETD_ERR_NONFINITE",
    -7: "ETD_ERR_TIMEOUT",
}
REACTIONS = {"none": 0, "logistic": 1, "logistic_ak": 2, "competition": 3}
TRACE_MAX = 64


class EtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRORS.get(code, str(code)), msg))
        self.code = code
        self.name = _ERRORS.get(code, str(code))


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 4), ("lo", ctypes.c_double * 4),
                ("hi", ctypes.c_double * 4)]


class Params(ctypes.Structure):
    _fields_ = [("nspecies", ctypes.c_int), ("precision", ctypes.c_int), ("krylov_tol", ctypes.c_double),
                ("m_max", ctypes.c_int), ("reaction", ctypes.c_int), ("rp", ctypes.c_double * 4),
                ("mu", ctypes.c_double * 2), ("beta", ctypes.c_double * 2), ("adjoint", ctypes.c_int),
                ("scheme", ctypes.c_int), ("boundary_data", ctypes.c_int)]

SCHEMES = {"etd1": 1, "etd2": 2, "etd2rk": 3, "etd3rk": 4, "etd4rk": 5, "etd3": 6}


class StepStats(ctypes.Structure):
    _fields_ = [("ncomp", ctypes.c_int * 2), ("substeps", ctypes.c_int * 2), ("rejections", ctypes.c_int * 2),
                ("krylov_iters", ctypes.c_int * 2), ("trace_len", ctypes.c_int * 2),
                ("trace_m", (ctypes.c_int * TRACE_MAX) * 2), ("trace_tau", (ctypes.c_double * TRACE_MAX) * 2)]

    def as_dict(self, nspecies=1):
        out = []
        for s in range(nspecies):
            n = self.trace_len[s]
            out.append({
                "ncomp": self.ncomp[s], "substeps": self.substeps[s], "rejections": self.rejections[s],
                "krylov_iters": self.krylov_iters[s],
                "trace": [(self.trace_tau[s][i], self.trace_m[s][i]) for i in range(n)],
            })
        return out


_LIB = None


def library():
    """Load the library (it must have been built, see build.py)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libetd_gb300.so is not built (run paper_2209_15095_gb300/build.py)")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "etd_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Params)]),
        "etd_create": (I, [ctypes.POINTER(Grid), ctypes.POINTER(Params), P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "etd_destroy": (None, [P]),
        "etd_init_domain": (I, [P, I, P, P]),
        "etd_step": (I, [P, D, ctypes.POINTER(P), ctypes.POINTER(StepStats)]),
        "etd_phi_combination": (I, [P, I, D, P, P, P, P, ctypes.POINTER(StepStats)]),
        "etd_phi_combination3": (I, [P, I, D, P, P, P, P, P, ctypes.POINTER(StepStats)]),
        "etd_apply_operator": (I, [P, I, D, P, P]),
        "etd_set_reaction": (I, [P, I, ctypes.POINTER(D)]),
        "etd_step_explicit": (I, [P, I, D, P, P, P, ctypes.POINTER(StepStats)]),
        "etd_adjoint_step": (I, [P, I, D, P, P, I, P, P, P, P, I]),
        "levelset_advance": (I, [P, I, P, P, D, I]),
        "levelset_prepare": (I, [P, P, I]),
        "etd_sync": (I, [P]),
        "etd_set_wait_limit": (I, [P, D]),
        "etd_selfcheck_round_f32": (I, [P, P, P, ctypes.c_longlong, P]),
        "etd_last_stats": (I, [P, ctypes.POINTER(StepStats)]),
        "levelset_last_stats": (I, [P, ctypes.POINTER(I)]),
        "etd_read_domain": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), P, P, P, I]),
        "etd_last_error": (ctypes.c_char_p, [P]),
        "etd_set_source": (I, [P, I, P, P]),
        "etd_boundary_points": (I, [P, I, P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "etd_set_boundary_values": (I, [P, I, P, P]),
        "etd_poisson_solve": (I, [P, I, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _ptr(t, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def selfcheck_round_f32(x):
    """The library's FP64 -> FP32 rounding (round to nearest, ties to even,
    on the integer pipe) and the hardware conversion of every element of x
    (a contiguous float64 CUDA tensor): returns (lib, hw), two float32 tensors
    of x's shape."""
    xp = _ptr(x, name="x")
    lib_out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    hw_out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    rc = library().etd_selfcheck_round_f32(xp, ctypes.c_void_p(lib_out.data_ptr()), ctypes.c_void_p(hw_out.data_ptr()),
                                           x.numel(), stream)
    if rc != 0:
        raise EtdError(rc, "etd_selfcheck_round_f32 failed")
    return lib_out, hw_out


class Context:
    """One library context: grid, parameters, workspace and stream."""

    def __init__(self, n, lo, hi, nspecies=1, precision="fp64", tol=1e-8, m_max=30, reaction="logistic",
                 rparams=(), mu=(1.0, 1.0), beta=(1.0, 1.0), device=None, adjoint=False, scheme="etd2",
                 boundary_data=False):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = library()
        self.n = tuple(int(v) for v in n)
        self.ndim = len(self.n)
        self.nspecies = nspecies
        self.device = torch.device(device or "cuda")
        g = Grid()
        g.ndim = self.ndim
        for d in range(self.ndim):
            g.n[d] = self.n[d]
            g.lo[d] = float(lo[d])
            g.hi[d] = float(hi[d])
        p = Params()
        p.nspecies = nspecies
        p.precision = {"fp64": 0, "mixed": 1}[precision]
        p.scheme = SCHEMES[scheme]
        p.krylov_tol = float(tol)
        p.m_max = int(m_max)
        p.reaction = REACTIONS[reaction]
        for i, v in enumerate(rparams):
            p.rp[i] = float(v)
        p.adjoint = 1 if adjoint else 0
        p.boundary_data = 1 if boundary_data else 0
        for s in range(2):
            p.mu[s] = float(mu[s] if s < len(mu) else mu[-1])
            p.beta[s] = float(beta[s] if s < len(beta) else beta[-1])
        self.grid_c, self.params_c = g, p
        nbytes = self.lib.etd_workspace_bytes(ctypes.byref(g), ctypes.byref(p))
        if nbytes == 0:
            raise EtdError(-1, "invalid grid or parameters")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        rc = self.lib.etd_create(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(aligned), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if rc != ETD_OK:
            raise EtdError(rc, "etd_create failed")
        self.ctx = ctx
        self._beta_fields = [None, None]
        self._sources = [(None, None), (None, None)]  # the library reads them during steps
        self._bvalues = [(None, None), (None, None)]
        self.adjoint_enabled = bool(adjoint)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            self.lib.etd_destroy(ctx)
            self.ctx = None

    def _check(self, rc):
        if rc != ETD_OK:
            raise EtdError(rc, self.lib.etd_last_error(self.ctx).decode())

    def init_domain(self, species, phi, beta_field=None):
        self._beta_fields[species] = beta_field  # the library reads it until the next init
        self._check(self.lib.etd_init_domain(self.ctx, species, _ptr(phi, self.n, "phi"),
                                             _ptr(beta_field, self.n, "beta_field")))

    def step(self, dt, us, stats=False):
        arr = (ctypes.c_void_p * 2)()
        for s, u in enumerate(us):
            arr[s] = _ptr(u, self.n, "u").value
        st = StepStats() if stats else None
        self._check(self.lib.etd_step(self.ctx, float(dt), arr, ctypes.byref(st) if st is not None else None))
        return st.as_dict(self.nspecies) if st is not None else None

    def phi_combination(self, species, dt, v0, v1, v2, y, stats=False):
        st = StepStats() if stats else None
        self._check(self.lib.etd_phi_combination(self.ctx, species, float(dt), _ptr(v0, self.n, "v0"),
                                                 _ptr(v1, self.n, "v1"), _ptr(v2, self.n, "v2"),
                                                 _ptr(y, self.n, "y"),
                                                 ctypes.byref(st) if st is not None else None))
        return st.as_dict(1)[0] if st is not None else None

    def phi_combination3(self, species, dt, v0, v1, v2, v3, y, stats=False):
        st = StepStats() if stats else None
        self._check(self.lib.etd_phi_combination3(self.ctx, species, float(dt), _ptr(v0, self.n, "v0"),
                                                  _ptr(v1, self.n, "v1"), _ptr(v2, self.n, "v2"),
                                                  _ptr(v3, self.n, "v3"), _ptr(y, self.n, "y"),
                                                  ctypes.byref(st) if st is not None else None))
        return st.as_dict(1)[0] if st is not None else None

    def poisson_solve(self, species, f, u, tol=1e-12, max_iter=100000):
        """Solve div(beta grad u) = f on the computational points (boundary data
        from set_boundary_values); u holds the initial guess and receives the
        solution.  Returns (iterations, relative residual)."""
        it, res = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.lib.etd_poisson_solve(self.ctx, species, _ptr(f, self.n, "f"), _ptr(u, self.n, "u"),
                                               float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

    def set_source(self, species, src_n, src_np1=None):
        """Additive source of F (full grid FP64) at t_n and, for ETD2RK's
        second stage, at t_n + dt (None: src_n).  None clears."""
        self._sources[species] = (src_n, src_np1)
        self._check(self.lib.etd_set_source(self.ctx, species, _ptr(src_n, self.n, "src_n"),
                                            _ptr(src_np1, self.n, "src_np1")))

    def boundary_points(self, species):
        """Boundary-data slot points of the current domain as a (ncomp, slots,
        N) float64 CUDA tensor (NaN where a slot is empty)."""
        n, sl = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.etd_boundary_points(self.ctx, species, None, ctypes.byref(n), ctypes.byref(sl)))
        out = torch.empty((max(n.value, 1), sl.value, self.ndim), dtype=torch.float64, device=self.device)
        self._check(self.lib.etd_boundary_points(self.ctx, species, ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.byref(n), ctypes.byref(sl)))
        return out[:n.value]

    def set_boundary_values(self, species, values_n, values_np1=None):
        """Boundary values at the slot points ((ncomp, slots) float64 CUDA
        tensors, t_n and t_n + dt).  None clears."""
        for v, name in ((values_n, "values_n"), (values_np1, "values_np1")):
            if v is not None and (not v.is_cuda or v.dtype != torch.float64 or not v.is_contiguous()):
                raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
        self._bvalues[species] = (values_n, values_np1)
        self._check(self.lib.etd_set_boundary_values(
            self.ctx, species, ctypes.c_void_p(values_n.data_ptr()) if values_n is not None else None,
            ctypes.c_void_p(values_np1.data_ptr()) if values_np1 is not None else None))

    def set_reaction(self, reaction, rparams):
        rp = (ctypes.c_double * 4)(*([float(v) for v in rparams] + [0.0] * (4 - len(rparams))))
        self._check(self.lib.etd_set_reaction(self.ctx, REACTIONS[reaction], rp))

    def step_explicit(self, species, dt, u_n, u_nm1, u_out, stats=False):
        st = StepStats() if stats else None
        self._check(self.lib.etd_step_explicit(self.ctx, species, float(dt), _ptr(u_n, self.n, "u_n"),
                                               _ptr(u_nm1, self.n, "u_nm1"), _ptr(u_out, self.n, "u_out"),
                                               ctypes.byref(st) if st is not None else None))
        return st.as_dict(1)[0] if st is not None else None

    def adjoint_step(self, species, dt, u_n, u_nm1, first, lam, acc, grad_beta, grad_params, nquad=8):
        gp = grad_params
        if not (isinstance(gp, torch.Tensor) and gp.is_cuda and gp.dtype == torch.float64 and gp.numel() >= 1):
            raise TypeError("grad_params must be a CUDA float64 tensor")
        self._check(self.lib.etd_adjoint_step(self.ctx, species, float(dt), _ptr(u_n, self.n, "u_n"),
                                              _ptr(u_nm1, self.n, "u_nm1"), 1 if first else 0,
                                              _ptr(lam, self.n, "lam"), _ptr(acc, self.n, "acc"),
                                              _ptr(grad_beta, self.n, "grad_beta"), ctypes.c_void_p(gp.data_ptr()),
                                              int(nquad)))

    def apply_operator(self, species, dt, x, y):
        self._check(self.lib.etd_apply_operator(self.ctx, species, float(dt), _ptr(x, self.n, "x"),
                                                _ptr(y, self.n, "y")))

    def levelset_advance(self, species, phi, u, dt, reinit):
        self._check(self.lib.levelset_advance(self.ctx, species, _ptr(phi, self.n, "phi"), _ptr(u, self.n, "u"),
                                              float(dt), 1 if reinit else 0))

    def levelset_prepare(self, phi, reinit):
        self._check(self.lib.levelset_prepare(self.ctx, _ptr(phi, self.n, "phi"), 1 if reinit else 0))

    def last_stats(self):
        st = StepStats()
        self._check(self.lib.etd_last_stats(self.ctx, ctypes.byref(st)))
        return st.as_dict(self.nspecies)

    def levelset_last_stats(self):
        info = (ctypes.c_int * 8)()
        self._check(self.lib.levelset_last_stats(self.ctx, info))
        return {"list": info[0], "tube": info[1], "nsub": info[2], "reinit_list": info[3], "reinit_tube": info[4],
                "reinit": info[5]}

    def sync(self):
        self._check(self.lib.etd_sync(self.ctx))

    def set_wait_limit(self, seconds):
        """Limit of every bounded device wait of later launches (<= 0: the
        default 1 s); a wait that reaches it is reported as ETD_ERR_TIMEOUT."""
        self._check(self.lib.etd_set_wait_limit(self.ctx, float(seconds)))

    def read_domain(self, species, arrays=True):
        import numpy as np
        size = 1
        for v in self.n:
            size *= v
        ncomp, nclamp, gersh = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        kind = np.zeros(size, dtype=np.uint8) if arrays else None
        idx = np.zeros(size, dtype=np.int32) if arrays else None
        diag = np.zeros(size, dtype=np.float64) if arrays else None
        rc = self.lib.etd_read_domain(
            self.ctx, species, ctypes.byref(ncomp), ctypes.byref(nclamp), ctypes.byref(gersh),
            kind.ctypes.data_as(ctypes.c_void_p) if arrays else None,
            idx.ctypes.data_as(ctypes.c_void_p) if arrays else None,
            diag.ctypes.data_as(ctypes.c_void_p) if arrays else None, size if arrays else 0)
        self._check(rc)
        out = {"ncomp": ncomp.value, "nclamp": nclamp.value, "gersh": gersh.value}
        if arrays:
            out["kind"] = kind.reshape(self.n)
            out["idx"] = idx[:ncomp.value].copy()
            out["diag"] = diag[:ncomp.value].copy()
        return out
