"""Seeded synthetic inputs for the workloads (initial level sets, initial
densities, diffusion fields).  This module holds none of the method's
arithmetic: it only draws numbers and evaluates the closed-form initial data,
and is the one module that both the CUDA path's callers and the oracle's
tests read.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) with
uniform = (x >> 11) * 2^-53, Gaussians by Box-Muller.

Workloads (the paper's experiments are 2D; the 3D/4D ones below are shaped
like them: a spreading species inside a level-set domain on a node grid):
  disc2d         64^2 on [-4,4]^2, phi0 = r - 1, u0 = cos(pi r / 2) inside
  star3d         128^3 on [-6,6]^3, star-shaped r0 = 1.5 (1 + 0.2 Y), Y a seeded
                 combination of real spherical harmonics of degree <= 4
                 normalised to max|Y| = 1; u0 = (1 - r/r0)(0.5 + 0.5 U), U
                 uniform noise smoothed by 3 damped Jacobi sweeps
  twoball3d      256^3 on [-8,8]^3, balls of radius 1.5 at (-2,0,0) and (2,0,0)
  adjoint_ball3d 128^3 on [-6,6]^3, fixed ball r = 4, beta = 1 + 0.3 g with g a
                 seeded Gaussian random field (correlation length 1)
  ellipsoid4d    48^4 on [-5,5]^4, semi-axes (1.5, 1.2, 1, 1)
  ball512        512^3 on [-8,8]^3, fixed ball r = 7 (bandwidth stress shape)
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed, count):
    """count successive SplitMix64 outputs from `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed, count):
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed, count):
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = np.maximum(u[0::2], 2.0 ** -53)
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
    return z[:count]


def grid_axes(n, lo, hi):
    return [lo[d] + (hi[d] - lo[d]) / (n[d] - 1) * np.arange(n[d], dtype=np.float64) for d in range(len(n))]


def grid_coords(n, lo, hi):
    return np.meshgrid(*grid_axes(n, lo, hi), indexing="ij")


def _legendre_assoc(l, m, x):
    """Associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase."""
    pmm = np.ones_like(x)
    if m > 0:
        s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * s
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def real_sph_harm(l, m, theta, phi):
    """Orthonormal real spherical harmonic Y_lm(theta, phi)."""
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    p = _legendre_assoc(l, am, np.cos(theta))
    if m == 0:
        return norm * p
    if m > 0:
        return math.sqrt(2.0) * norm * p * np.cos(m * phi)
    return math.sqrt(2.0) * norm * p * np.sin(am * phi)


def star_radius_fn(seed=1, lmax=4):
    coef = 2.0 * uniform(seed, (lmax + 1) ** 2) - 1.0
    terms = [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1)]

    def Y(theta, phi):
        out = np.zeros(np.broadcast(theta, phi).shape)
        for c, (l, m) in zip(coef, terms):
            out = out + c * real_sph_harm(l, m, theta, phi)
        return out

    th = np.linspace(0.0, math.pi, 721)
    ph = np.arange(1440) * (2.0 * math.pi / 1440)
    T, P = np.meshgrid(th, ph, indexing="ij")
    ymax = float(np.max(np.abs(Y(T, P))))

    def r0(theta, phi):
        return 1.5 * (1.0 + 0.2 * Y(theta, phi) / ymax)

    return r0


def jacobi_smooth(U, sweeps=3):
    """U <- U + (2/3)(mean of the available axis neighbours - U), `sweeps` times."""
    for _ in range(sweeps):
        acc = np.zeros_like(U)
        cnt = np.zeros_like(U)
        for d in range(U.ndim):
            for s in (-1, 1):
                sl_dst = [slice(None)] * U.ndim
                sl_src = [slice(None)] * U.ndim
                if s > 0:
                    sl_dst[d], sl_src[d] = slice(0, -1), slice(1, None)
                else:
                    sl_dst[d], sl_src[d] = slice(1, None), slice(0, -1)
                acc[tuple(sl_dst)] += U[tuple(sl_src)]
                cnt[tuple(sl_dst)] += 1.0
        U = U + (2.0 / 3.0) * (acc / cnt - U)
    return U


def gaussian_field(n, h, seed=3, corr=1.0):
    """White noise convolved separably with a Gaussian of standard deviation
    corr/sqrt(2) (so the field's covariance is exp(-r^2/(2 corr^2))), kernel
    truncated at 4 sigma, zero padding; normalised to zero mean and unit
    standard deviation, clipped to [-1, 1]."""
    g = gaussian(seed, int(np.prod(n))).reshape(n)
    sig = corr / math.sqrt(2.0) / h
    half = int(math.ceil(4.0 * sig))
    x = np.arange(-half, half + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sig) ** 2)
    k /= k.sum()
    for d in range(len(n)):
        g = np.apply_along_axis(lambda a: np.convolve(a, k, mode="same"), d, g)
    g = (g - g.mean()) / g.std()
    return np.clip(g, -1.0, 1.0)


class Workload:
    """Initial data of one workload: grid (n, lo, hi), per-species phi0 / u0,
    beta (scalar or node field), mu, reaction, parameters, time step."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    @property
    def h(self):
        return (self.hi[0] - self.lo[0]) / (self.n[0] - 1)


def disc2d(n=64):
    lo, hi = (-4.0, -4.0), (4.0, 4.0)
    x, y = grid_coords((n, n), lo, hi)
    r = np.sqrt(x * x + y * y)
    phi0 = r - 1.0
    u0 = np.where(phi0 < 0, np.cos(math.pi * r / 2.0), 0.0)
    return Workload(name="disc2d", n=(n, n), lo=lo, hi=hi, phi0=[phi0], u0=[u0], beta=[1.0], mu=[2.0],
                    reaction="logistic", rparams=(), dt=1e-2, steps=100, tol=1e-8, m_max=30,
                    reinit_every=5, reinit_at_start=False)


def star3d(n=128, seed_shape=1, seed_noise=2, box=6.0):
    lo, hi = (-box,) * 3, (box,) * 3
    x, y, z = grid_coords((n, n, n), lo, hi)
    r = np.sqrt(x * x + y * y + z * z)
    theta = np.arccos(np.clip(np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0), -1.0, 1.0))
    ph = np.arctan2(y, x)
    r0 = star_radius_fn(seed_shape)(theta, ph)
    phi0 = r - r0
    U = jacobi_smooth(uniform(seed_noise, n ** 3).reshape(n, n, n), 3)
    u0 = np.where(phi0 < 0, (1.0 - r / r0) * (0.5 + 0.5 * U), 0.0)
    return Workload(name="star3d", n=(n, n, n), lo=lo, hi=hi, phi0=[phi0], u0=[u0], beta=[1.0], mu=[1.0],
                    reaction="logistic", rparams=(), dt=5e-3, steps=400, tol=1e-7, tol_mixed=1e-5, m_max=40,
                    reinit_every=5, reinit_at_start=True)


def twoball3d(n=256):
    lo, hi = (-8.0,) * 3, (8.0,) * 3
    x, y, z = grid_coords((n, n, n), lo, hi)
    phis, us = [], []
    for cx in (-2.0, 2.0):
        r = np.sqrt((x - cx) ** 2 + y * y + z * z)
        p = r - 1.5
        phis.append(p)
        us.append(np.where(p < 0, np.cos(math.pi * r / 3.0), 0.0))
    return Workload(name="twoball3d", n=(n, n, n), lo=lo, hi=hi, phi0=phis, u0=us, beta=[1.0, 0.5],
                    mu=[1.0, 0.8], reaction="competition", rparams=(0.5, 0.8, 1.2), dt=5e-3, steps=200,
                    tol=1e-5, m_max=40, reinit_every=5, reinit_at_start=False)


def adjoint_ball3d(n=128, seed=3):
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    x, y, z = grid_coords((n, n, n), lo, hi)
    r = np.sqrt(x * x + y * y + z * z)
    phi0 = r - 4.0
    h = 12.0 / (n - 1)
    g = gaussian_field((n, n, n), h, seed=seed)
    beta = 1.0 + 0.3 * g
    u0 = np.where(phi0 < 0, np.cos(math.pi * r / 8.0), 0.0)
    return Workload(name="adjoint_ball3d", n=(n, n, n), lo=lo, hi=hi, phi0=[phi0], u0=[u0], beta=[beta],
                    mu=[0.0], reaction="logistic_ak", rparams=(1.0, 1.0), rparams_target=(1.1, 1.0),
                    beta_target_scale=1.05, dt=1e-2, steps=100, tol=1e-7, m_max=40, checkpoint_every=10)


def ellipsoid4d(n=48):
    lo, hi = (-5.0,) * 4, (5.0,) * 4
    xs = grid_coords((n,) * 4, lo, hi)
    a = (1.5, 1.2, 1.0, 1.0)
    rho = np.sqrt(sum((xs[d] / a[d]) ** 2 for d in range(4)))
    phi0 = min(a) * (rho - 1.0)
    u0 = np.where(phi0 < 0, np.cos(math.pi * rho / 2.0), 0.0)
    return Workload(name="ellipsoid4d", n=(n,) * 4, lo=lo, hi=hi, phi0=[phi0], u0=[u0], beta=[1.0], mu=[1.0],
                    reaction="logistic", rparams=(), dt=5e-3, steps=100, tol=1e-5, m_max=40, reinit_every=5,
                    reinit_at_start=True)


def ball512(n=512, radius=7.0, box=8.0):
    lo, hi = (-box,) * 3, (box,) * 3
    ax = grid_axes((n, n, n), lo, hi)
    x = ax[0][:, None, None]
    y = ax[1][None, :, None]
    z = ax[2][None, None, :]
    r = np.sqrt(x * x + y * y + z * z)
    phi0 = r - radius
    u0 = np.where(phi0 < 0, np.cos(math.pi * r / (2.0 * radius)), 0.0)
    return Workload(name="ball512", n=(n, n, n), lo=lo, hi=hi, phi0=[phi0], u0=[u0], beta=[1.0], mu=[0.0],
                    reaction="logistic", rparams=(), dt=1e-2, steps=10, tol=1e-7, m_max=40)


def fixed_ball(n, box, radius, ndim=3, beta=1.0):
    """Fixed ball (or disc) domain of a given radius, for parity cases."""
    lo, hi = (-box,) * ndim, (box,) * ndim
    xs = grid_coords((n,) * ndim, lo, hi)
    r = np.sqrt(sum(c * c for c in xs))
    phi0 = r - radius
    u0 = np.where(phi0 < 0, np.cos(math.pi * r / (2.0 * radius)), 0.0)
    return Workload(name="fixed_ball%dd" % ndim, n=(n,) * ndim, lo=lo, hi=hi, phi0=[phi0], u0=[u0],
                    beta=[beta], mu=[0.0], reaction="logistic", rparams=(), dt=1e-2, steps=1, tol=1e-8, m_max=40)


def virus_radius_fn(samples=200001):
    """Boundary of the virus-shaped domain of Sec. 4.1, x = (0.6 + 0.1 sin 12t)
    cos t, y = (0.6 + 0.05 sin 12t) sin t, as a radius R(psi) of the polar
    angle (the curve's polar angle increases strictly with t), interpolated
    periodically from a dense sampling."""
    t = np.linspace(0.0, 2.0 * math.pi, samples)
    x = (0.6 + 0.1 * np.sin(12 * t)) * np.cos(t)
    y = (0.6 + 0.05 * np.sin(12 * t)) * np.sin(t)
    psi = np.unwrap(np.arctan2(y, x))
    r = np.hypot(x, y)

    def R(ang):
        a = np.mod(ang - psi[0], 2.0 * math.pi) + psi[0]
        return np.interp(a, psi, r)

    return R


def virus_exact(x, y):
    """Exact solution u = e^x (x^2 sin y + y^2) of the Sec. 4.1 example."""
    return np.exp(x) * (x * x * np.sin(y) + y * y)


def virus_beta(x, y):
    return 2.0 + np.sin(x * y)


def virus_source(x, y):
    """f = div(beta grad u) for the exact u and beta = 2 + sin(xy):
    beta Lap u + grad beta . grad u, with Lap u = e^x (y^2 + 4x sin y + 2 sin y + 2)."""
    ex = np.exp(x)
    ux = ex * (x * x * np.sin(y) + y * y + 2 * x * np.sin(y))
    uy = ex * (x * x * np.cos(y) + 2 * y)
    lap = ex * (y * y + 4 * x * np.sin(y) + 2 * np.sin(y) + 2)
    return virus_beta(x, y) * lap + y * np.cos(x * y) * ux + x * np.cos(x * y) * uy


def virus2d(N=100):
    """(N+1)^2 node grid on [-1, 1]^2 with the virus domain (phi = r - R(psi) < 0
    inside), the beta node field, the source and the exact solution."""
    n = (N + 1, N + 1)
    lo, hi = (-1.0, -1.0), (1.0, 1.0)
    x, y = grid_coords(n, lo, hi)
    R = virus_radius_fn()
    phi = np.hypot(x, y) - R(np.arctan2(y, x))
    return Workload(name="virus2d", n=n, lo=lo, hi=hi, phi0=[phi], u0=[virus_exact(x, y)], beta=[1.0], mu=[0.0],
                    reaction="none", rparams=(), dt=0.0, steps=0, tol=1e-12, m_max=40,
                    beta_field=virus_beta(x, y), source=virus_source(x, y), exact=virus_exact)
