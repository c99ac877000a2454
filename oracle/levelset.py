"""Level-set step of the free-boundary algorithm (Sec. 4.3, Algorithm Steps 1-2;
Stefan condition of Eq. free and Sec. 4.3: normal speed mu |grad u|).

The paper names the methods and prints no formulas; the readings below are
published methods restated, with the constants this implementation uses.

Local level set (Peng, Merriman, Osher, Zhao & Kang 1999, cited by the paper):
  phi is kept clamped to [-G, G], G = 6h.  The tube S = {|phi| < G}; the
  update set T is S grown by one node along every axis.  Nodes outside T are
  not updated.  Out-of-box neighbours repeat the edge value.
Extension of u (Aslam 2004 quadratic extrapolation in the normal direction):
  n = grad phi / |grad phi| (central differences, |grad phi| floored at 1e-12).
  valid0 = computational points, valid1 = valid0 nodes whose 2N neighbours
  are valid0, valid2 likewise from valid1.  u_n = n . grad u (central) on
  valid1, u_nn = n . grad u_n on valid2.  Then three pseudo-time sweeps of
  q_tau + n . grad q = s, first-order upwind in the direction of n, forward
  Euler with step h/(2 sqrt N), ceil(12 sqrt N) steps (pseudo-time >= 6h):
  u_nn (s = 0) on T minus valid2, then u_n (s = u_nn) on T minus valid1, then
  u (s = u_n) on T minus valid0.  Unknown values start at 0.
Stefan speed (closest-point extension): at every node of T,
  x_G = x - phi n, V = mu max(0, (4 u(x_G - h n) - u(x_G - 2h n)) / (2h))
  with N-linear interpolation of the extended u (sample points clamped to
  the box); V = 0 off T.
Advection phi_t + V |grad phi| = 0: Godunov Hamiltonian with HJ-WENO5
  one-sided derivatives (Jiang & Peng 2000; eps = 1e-6), Shu-Osher TVD-RK3,
  n_sub = max(1, ceil(dt max V N / (0.5 h))) equal substeps.
Reinitialisation phi_t + S(phi_0)(|grad phi| - 1) = 0, S = phi_0/sqrt(phi_0^2 + h^2)
  (Sussman, Smereka & Osher 1994), same spatial scheme with the Godunov
  upwinding chosen by the sign of S, TVD-RK3, pseudo-step 0.5h/sqrt N,
  ceil(12 sqrt N) steps, T fixed from phi_0.
After advection and after reinitialisation phi is clamped to [-G, G].
"""
import math

import numpy as np

from .grid import shift_clamped

BAND = 6.0          # G / h
WENO_EPS = 1e-6
GRAD_FLOOR = 1e-12


def pseudo_steps(ndim):
    return int(math.ceil(12.0 * math.sqrt(ndim)))


def tube(phi, h):
    """Update set T: {|phi| < G} grown by one node along every axis."""
    s = np.abs(phi) < BAND * h
    t = s.copy()
    for d in range(phi.ndim):
        t |= shift_clamped(s, d, 1) | shift_clamped(s, d, -1)
    return t


def _weno(v1, v2, v3, v4, v5):
    """HJ-WENO5 one-sided derivative from the five divided differences."""
    p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
    p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
    p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
    s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2
    s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
    a1 = 0.1 / (WENO_EPS + s1) ** 2
    a2 = 0.6 / (WENO_EPS + s2) ** 2
    a3 = 0.3 / (WENO_EPS + s3) ** 2
    return (a1 * p1 + a2 * p2 + a3 * p3) / (a1 + a2 + a3)


def weno_derivatives(phi, h, d):
    """(D-, D+) along axis d: WENO5 backward / forward derivatives."""
    q = {}
    for k in range(-2, 4):
        # q[k] = (phi_{i+k} - phi_{i+k-1}) / h
        q[k] = (shift_clamped(phi, d, k) - shift_clamped(phi, d, k - 1)) / h
    dm = _weno(q[-2], q[-1], q[0], q[1], q[2])
    dp = _weno(q[3], q[2], q[1], q[0], q[-1])
    return dm, dp


def godunov_grad(phi, h, positive):
    """Godunov |grad phi| for a Hamiltonian s |grad phi| with s > 0 where
    `positive` is True (outward motion) and s < 0 elsewhere."""
    acc = np.zeros_like(phi)
    for d in range(phi.ndim):
        a, b = weno_derivatives(phi, h, d)
        pos = np.maximum(np.maximum(a, 0.0) ** 2, np.minimum(b, 0.0) ** 2)
        neg = np.maximum(np.minimum(a, 0.0) ** 2, np.maximum(b, 0.0) ** 2)
        acc += np.where(positive, pos, neg)
    return np.sqrt(acc)


def _rk3(phi, L, dt, T):
    """Shu-Osher TVD-RK3 restricted to the update set T."""
    p1 = np.where(T, phi + dt * L(phi), phi)
    p2 = np.where(T, 0.75 * phi + 0.25 * (p1 + dt * L(p1)), phi)
    return np.where(T, phi / 3.0 + 2.0 / 3.0 * (p2 + dt * L(p2)), phi)


def normals(phi, h):
    g = [(shift_clamped(phi, d, 1) - shift_clamped(phi, d, -1)) / (2.0 * h) for d in range(phi.ndim)]
    nrm = np.maximum(np.sqrt(sum(x * x for x in g)), GRAD_FLOOR)
    return [x / nrm for x in g]


def _all_nb(mask):
    out = mask.copy()
    for d in range(mask.ndim):
        out &= shift_clamped(mask, d, 1) & shift_clamped(mask, d, -1)
    return out


def _n_dot_grad_central(q, n, h):
    return sum(n[d] * (shift_clamped(q, d, 1) - shift_clamped(q, d, -1)) / (2.0 * h) for d in range(q.ndim))


def _n_dot_grad_upwind(q, n, h):
    acc = np.zeros_like(q)
    for d in range(q.ndim):
        back = (q - shift_clamped(q, d, -1)) / h
        fwd = (shift_clamped(q, d, 1) - q) / h
        acc += n[d] * np.where(n[d] > 0.0, back, fwd)
    return acc


def _sweep(q, src, n, h, region):
    ndim = q.ndim
    dtau = h / (2.0 * math.sqrt(ndim))
    q = np.where(region, 0.0, q)
    for _ in range(pseudo_steps(ndim)):
        q = np.where(region, q - dtau * (_n_dot_grad_upwind(q, n, h) - src), q)
    return q


def extend(u, phi, comp, h, T=None):
    """Aslam quadratic normal extrapolation of u from the computational points
    into T minus the computational points."""
    if T is None:
        T = tube(phi, h)
    n = normals(phi, h)
    v0 = comp
    v1 = _all_nb(v0)
    v2 = _all_nb(v1)
    u = np.where(v0, u, 0.0)
    un = np.where(v1, _n_dot_grad_central(u, n, h), 0.0)
    unn = np.where(v2, _n_dot_grad_central(un, n, h), 0.0)
    zero = np.zeros_like(u)
    unn = _sweep(unn, zero, n, h, T & ~v2)
    un = _sweep(un, unn, n, h, T & ~v1)
    return _sweep(u, un, n, h, T & ~v0)


def interp(a, lo, h, pts):
    """N-linear interpolation of node array a at points pts (..., N); points
    are clamped to the box."""
    N = a.ndim
    n = np.array(a.shape)
    s = (pts - lo) / h
    s = np.clip(s, 0.0, n - 1.0)
    i0 = np.minimum(np.floor(s).astype(np.int64), n - 2)
    f = s - i0
    out = np.zeros(pts.shape[:-1])
    for corner in range(1 << N):
        w = np.ones(pts.shape[:-1])
        idx = []
        for d in range(N):
            bit = (corner >> d) & 1
            w = w * (f[..., d] if bit else (1.0 - f[..., d]))
            idx.append(i0[..., d] + bit)
        out += w * a[tuple(idx)]
    return out


def stefan_speed(u_ext, phi, grid, mu, T):
    """V = mu |grad u| at the interface, carried to every node of T along the
    normal (closest-point extension)."""
    h = grid.h
    n = np.stack(normals(phi, h), axis=-1)
    x = np.stack(grid.coords(), axis=-1)
    xg = x - phi[..., None] * n
    u1 = interp(u_ext, grid.lo, h, xg - h * n)
    u2 = interp(u_ext, grid.lo, h, xg - 2.0 * h * n)
    V = mu * np.maximum(0.0, (4.0 * u1 - u2) / (2.0 * h))
    return np.where(T, V, 0.0)


def advect(phi, V, dt, h, T):
    N = phi.ndim
    vmax = float(np.max(np.where(T, V, 0.0)))
    nsub = max(1, int(math.ceil(dt * vmax * N / (0.5 * h))))
    dts = dt / nsub

    def L(p):
        return -V * godunov_grad(p, h, True)

    for _ in range(nsub):
        phi = _rk3(phi, L, dts, T)
    return phi, nsub


def reinit(phi, h):
    N = phi.ndim
    T = tube(phi, h)
    S = phi / np.sqrt(phi * phi + h * h)
    positive = S > 0.0
    dtau = 0.5 * h / math.sqrt(N)

    def L(p):
        return -S * (godunov_grad(p, h, positive) - 1.0)

    for _ in range(pseudo_steps(N)):
        phi = _rk3(phi, L, dtau, T)
    return clamp(phi, h)


def clamp(phi, h):
    return np.clip(phi, -BAND * h, BAND * h)


def levelset_advance(phi, u, comp, grid, dt, mu, do_reinit):
    """One level-set step: extend u, Stefan speed, advect, (reinitialise),
    clamp.  Returns (phi_new, u_extended, nsub)."""
    h = grid.h
    T = tube(phi, h)
    u_ext = extend(u, phi, comp, h, T)
    V = stefan_speed(u_ext, phi, grid, mu, T)
    phi_new, nsub = advect(phi, V, dt, h, T)
    phi_new = clamp(phi_new, h)
    if do_reinit:
        phi_new = reinit(phi_new, h)
    return phi_new, u_ext, nsub
