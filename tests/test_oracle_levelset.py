"""Pins for oracle.levelset and oracle.freeboundary: WENO5's fifth order and
exactness on linear data, Godunov |grad phi| = 1 on a distance function,
reinitialisation of a distance function leaving the interface in place,
Aslam extension converging and, on a planar front, quadratic rather than
linear (a negative control with u_nn dropped fails the bound), the Stefan speed of a unit-slope profile, the
advected circle's radius, and for the free-boundary disc: grid (D4) symmetry,
radial symmetry of the front, and a monotonically growing domain."""
import math

import numpy as np
import pytest

from oracle import levelset as ls
from oracle.eb import classify
from oracle.freeboundary import FreeBoundary, Species
from oracle.grid import Grid
from paper_2209_15095_gb300 import inputs


def test_weno5_fifth_order_and_linear_exact():
    errs = []
    for n in (41, 81):
        g = Grid((n, n), (-1, -1), (1, 1))
        x, y = g.coords()
        f = np.sin(2 * x) * np.cos(y)
        dm, dp = ls.weno_derivatives(f, g.h, 0)
        ex = 2 * np.cos(2 * x) * np.cos(y)
        sl = (slice(5, -5), slice(5, -5))
        errs.append(max(np.max(np.abs(dm - ex)[sl]), np.max(np.abs(dp - ex)[sl])))
    assert errs[0] / errs[1] > 24.0  # 2^5 = 32
    g = Grid((30, 30), (-1, -1), (1, 1))
    x, y = g.coords()
    for d, slope in ((0, 0.3), (1, -1.7)):
        f = 0.2 + 0.3 * x - 1.7 * y
        dm, dp = ls.weno_derivatives(f, g.h, d)
        sl = (slice(4, -4), slice(4, -4))
        assert np.allclose(dm[sl], slope, atol=1e-12) and np.allclose(dp[sl], slope, atol=1e-12)


def test_godunov_gradient_of_plane_distance():
    g = Grid((30, 30), (-1, -1), (1, 1))
    x, y = g.coords()
    nx, ny = 0.6, -0.8
    f = nx * x + ny * y - 0.1
    for positive in (True, False):
        G = ls.godunov_grad(f, g.h, positive)
        assert np.allclose(G[4:-4, 4:-4], 1.0, atol=1e-12)


def _crossing_x(row, xs):
    i = np.where((row[:-1] < 0) & (row[1:] >= 0))[0][-1]
    return xs[i] - row[i] * (xs[i + 1] - xs[i]) / (row[i + 1] - row[i])


def test_reinit_keeps_distance_interface():
    g = Grid((64, 64), (-4, -4), (4, 4))
    r = g.radius(center=(0.013, -0.021))
    ph = ls.clamp(r - 1.5, g.h)
    ph2 = ls.reinit(ph, g.h)
    xs = g.axis(1)
    for row in (30, 32, 34):
        assert abs(_crossing_x(ph2[row], xs) - _crossing_x(ph[row], xs)) < 1e-2 * g.h
    band = np.abs(r - 1.5) < 3 * g.h
    assert np.max(np.abs(ph2 - ph)[band]) < 1e-2 * g.h


def test_extension_converges():
    errs = []
    for n in (64, 128):
        g = Grid((n, n), (-4, -4), (4, 4))
        r = g.radius()
        R = 1.5
        prof = (R - r) + 0.3 * (R - r) ** 2
        _, _, comp = classify(g, r - R)
        ph = ls.clamp(r - R, g.h)
        ue = ls.extend(np.where(comp, prof, 0.0), ph, comp, g.h)
        near = (np.abs(r - R) < 2.5 * g.h) & ~comp
        errs.append(np.max(np.abs(ue - prof)[near]))
    assert errs[1] < errs[0] / 1.5


def _planar_extension(n, ndim, prof_ab, drop_unn):
    """Extension of u = a d + b d^2 across the planar face x = X0 of a box
    domain (x the last axis, d = X0 - |x| the distance inside); returns the
    errors of the extended u at the first two nodes beyond the computational
    set on the middle line, in units of b h^2."""
    a, b = prof_ab
    X0 = 0.5123
    g = Grid((n,) * ndim, (-1.0,) * ndim, (1.0,) * ndim)
    x = g.coords()
    phi = np.abs(x[-1]) - X0
    for dd in range(ndim - 1):
        phi = np.maximum(phi, np.abs(x[dd]) - 0.6)
    d = X0 - np.abs(x[-1])
    prof = a * d + b * d * d
    _, _, comp = classify(g, phi)
    ph = ls.clamp(phi, g.h)
    T = ls.tube(ph, g.h)
    u = np.where(comp, prof, 0.0)
    if not drop_unn:
        ue = ls.extend(u, ph, comp, g.h, T)
    else:
        # negative control built here, not in the oracle: linear
        # extrapolation (the u_nn sweep dropped, u_nn = 0)
        nrm = ls.normals(ph, g.h)
        v1 = ls._all_nb(comp)
        un = np.where(v1, ls._n_dot_grad_central(u, nrm, g.h), 0.0)
        un = ls._sweep(un, np.zeros_like(u), nrm, g.h, T & ~v1)
        ue = ls._sweep(u, un, nrm, g.h, T & ~comp)
    mid = (n // 2,) * (ndim - 1)
    i0 = int(np.where(comp[mid])[0].max())
    return [(ue[mid + (i0 + k,)] - prof[mid + (i0 + k,)]) / (b * g.h * g.h) for k in (1, 2)]


@pytest.mark.parametrize("ndim,n", [(2, 41), (2, 81), (2, 161), (3, 41)])
def test_extension_quadratic_planar_front(ndim, n):
    """Aslam's quadratic extrapolation (Sec. 4.3, Step 2) on a planar front
    with the normal along a grid axis.  Central differences of a quadratic
    are exact, so u_n = u' and u_nn = u'' = 2b on their valid sets and the
    u_nn and u_n sweeps have exact steady states (a constant, a linear
    function).  The first-order upwind u sweep then gives
    q_i = q_{i-1} + h u'(x_i), while u(x_i) = u(x_{i-1}) + h u'(x_i) - b h^2:
    the k-th node beyond the computational set is off by k b h^2.  Linear
    extrapolation (u_nn dropped) freezes u_n at u'(x_{i0-1}) and is off by
    -(k^2 + 2k) b h^2.  The finite pseudo-time moves the first two nodes by
    less than 0.25 b h^2 (the linear variant by less than 0.7 b h^2), so
    |e_k - k b h^2| <= 0.5 b h^2 separates the two by more than 2 b h^2."""
    errs = _planar_extension(n, ndim, (0.5, 3.0), drop_unn=False)
    for k, e in zip((1, 2), errs):
        assert abs(e - k) <= 0.5, (k, e)
    lin = _planar_extension(n, ndim, (0.5, 3.0), drop_unn=True)
    for k, e in zip((1, 2), lin):
        assert abs(e - k) > 2.5, (k, e)
        assert abs(e + k * k + 2 * k) <= 1.0, (k, e)


def test_stefan_speed_unit_slope():
    g = Grid((64, 64), (-4, -4), (4, 4))
    r = g.radius()
    R, mu = 1.5, 2.0
    _, _, comp = classify(g, r - R)
    ph = ls.clamp(r - R, g.h)
    T = ls.tube(ph, g.h)
    ue = ls.extend(np.where(comp, R - r, 0.0), ph, comp, g.h, T)
    V = ls.stefan_speed(ue, ph, g, mu, T)
    band = np.abs(r - R) < 3 * g.h
    assert np.max(np.abs(V[band] - mu)) < 0.1 * mu
    assert np.all(V[~T] == 0.0)


def test_advection_constant_speed():
    g = Grid((80, 80), (-4, -4), (4, 4))
    r = g.radius()
    ph = ls.clamp(r - 1.0, g.h)
    T = ls.tube(ph, g.h)
    V = np.where(T, 1.0, 0.0)
    for _ in range(4):
        T = ls.tube(ph, g.h)
        ph, _ = ls.advect(ph, np.where(T, 1.0, 0.0), 0.05, g.h, T)
        ph = ls.clamp(ph, g.h)
    xs = g.axis(1)
    x0 = _crossing_x(ph[40], xs)
    # the front moved by V t = 0.2 from radius 1 (row 40 is y = 0.05)
    assert abs(math.sqrt(x0 ** 2 + xs[40] ** 2) - 1.2) < 0.02 * g.h * 10


@pytest.fixture(scope="module")
def disc_run():
    w = inputs.disc2d()
    g = Grid(w.n, w.lo, w.hi)
    fb = FreeBoundary(g, [Species(w.phi0[0], w.u0[0], 1.0, w.mu[0])], w.reaction, w.rparams, w.tol, w.m_max,
                      reinit_every=w.reinit_every)
    inside = [fb.sp[0].phi < 0]
    for _ in range(40):
        fb.step(w.dt)
        inside.append(fb.sp[0].phi < 0)
    return g, fb, inside


def test_free_boundary_grid_symmetry(disc_run):
    g, fb, _ = disc_run
    for a in (fb.sp[0].phi, fb.sp[0].u):
        scale = np.max(np.abs(a))
        for b in (a[::-1, :], a[:, ::-1], a.T):
            assert np.max(np.abs(a - b)) <= 1e-10 * scale


def test_free_boundary_monotone_growth_and_round(disc_run):
    g, fb, inside = disc_run
    for a, b in zip(inside[:-1], inside[1:]):
        assert np.all(b[a])  # nodes never leave the domain
    assert inside[-1].sum() > inside[0].sum()
    # interface radius along 16 rays (bilinear sampling of phi, bisection)
    ph = fb.sp[0].phi
    radii = []
    for k in range(16):
        th = 2 * math.pi * k / 16 + 0.1
        lo_r, hi_r = 0.5, 3.0
        for _ in range(50):
            mid = 0.5 * (lo_r + hi_r)
            p = np.array([[mid * math.cos(th), mid * math.sin(th)]])
            if ls.interp(ph, g.lo, g.h, p)[0] < 0:
                lo_r = mid
            else:
                hi_r = mid
        radii.append(lo_r)
    radii = np.array(radii)
    assert (radii.max() - radii.min()) / radii.mean() <= 0.05
    assert radii.mean() > 1.0
