"""Uniform node grid (Sec. 2: x_ij = (x_L + (i-1)h, y_L + (j-1)h)), generalised
to N axes.  Arrays are numpy arrays of shape ``n`` in C order, axis 0 slowest,
the last axis fastest.  The spacing h is the same on every axis.
"""
import numpy as np


class Grid:
    def __init__(self, n, lo, hi):
        self.n = tuple(int(v) for v in n)
        self.ndim = len(self.n)
        self.lo = np.asarray(lo, dtype=np.float64).reshape(self.ndim)
        self.hi = np.asarray(hi, dtype=np.float64).reshape(self.ndim)
        hs = (self.hi - self.lo) / (np.asarray(self.n, dtype=np.float64) - 1.0)
        if np.max(np.abs(hs - hs[0])) > 1e-12 * hs[0]:
            raise ValueError("grid spacing must be the same on every axis")
        self.h = float(hs[0])

    @property
    def size(self):
        return int(np.prod(self.n))

    def axis(self, d):
        """Node coordinates along axis d: lo_d + i h, i = 0..n_d-1."""
        return self.lo[d] + self.h * np.arange(self.n[d], dtype=np.float64)

    def coords(self):
        """List of N arrays (shape n) holding each node's coordinates."""
        return np.meshgrid(*[self.axis(d) for d in range(self.ndim)], indexing="ij")

    def radius(self, center=None):
        x = self.coords()
        c = np.zeros(self.ndim) if center is None else np.asarray(center, dtype=np.float64)
        return np.sqrt(sum((x[d] - c[d]) ** 2 for d in range(self.ndim)))


def shift(a, d, s, fill):
    """b[i] = a[i + s e_d]; entries whose source lies outside the box get `fill`."""
    b = np.full_like(a, fill)
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if s > 0:
        src[d] = slice(s, None)
        dst[d] = slice(0, -s)
    else:
        src[d] = slice(0, s)
        dst[d] = slice(-s, None)
    b[tuple(dst)] = a[tuple(src)]
    return b


def shift_clamped(a, d, s):
    """b[i] = a[clamp(i + s e_d)]: replicate the edge value past the box."""
    n = a.shape[d]
    idx = np.clip(np.arange(n) + s, 0, n - 1)
    return np.take(a, idx, axis=d)
