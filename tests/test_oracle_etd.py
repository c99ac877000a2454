"""Pins for oracle.etd: ETD2 and ETD2RK on a scalar ODE in closed form;
ETD3RK and ETD4RK exact for forcing quadratic in t, phi_0 alone for F = 0,
orders 3 and 4 on a Bernoulli ODE and on a stiff EB system;
first-order (ETD1) and second-order (ETD2, ETD2RK) convergence for a
manufactured solution on a fixed circle, and the paper's Table 1 (ETD2 and
ETD2RK on the peanut domain, Sec. 4.2.1) within a factor of 3; stability of
ETD2 on the same problem for steps up to dt = 0.1 (Sec. 4.2.2, Fig. 5)."""
import math
import os

import numpy as np
import pytest

from oracle import etd, phi
from oracle.eb import EBOperator
from oracle.grid import Grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_etd2.txt")
GOLDEN_RK = os.path.join(os.path.dirname(__file__), "golden", "table1_etd2rk.txt")


class _ScalarOp:
    def __init__(self, c):
        import scipy.sparse as sp
        self.C = sp.csr_matrix(np.array([[c]]))
        self.ncomp = 1

    def gershgorin(self):
        return abs(self.C[0, 0])


def test_etd2_scalar_closed_form():
    # u' = c u + F with F = a + b t: ETD2 is exact for F linear in t.
    c, a, b, dt = -3.0, 0.7, -1.3, 0.1
    op = _ScalarOp(c)
    u = np.array([0.4])
    exact = lambda t: (0.4 + (a / c + b / c ** 2)) * math.exp(c * t) - a / c - b / c ** 2 - b * t / c
    # step 1 from t = dt with F_n = a + b dt and F_{n-1} = a
    u1 = np.array([exact(dt)])
    u2, _ = etd.etd2_step(op, u1, np.array([a + b * dt]), np.array([a]), dt, tol=1e-13, m_max=5)
    assert abs(u2[0] - exact(2 * dt)) < 1e-13


def test_etd2rk_scalar_closed_form():
    # u' = c u + F with F = a + b t: ETD2RK is exact for F linear in t and
    # independent of u (the second stage adds dt^2 phi_2(c dt) b).
    c, a, b, dt, t0 = -3.0, 0.7, -1.3, 0.1, 0.2
    op = _ScalarOp(c)
    C0 = 0.4 + a / c + b / c ** 2
    exact = lambda t: C0 * math.exp(c * t) - a / c - b / c ** 2 - b * t / c
    F_of = lambda u, t: np.full_like(u, a + b * t)
    u1, a1, _ = etd.etd2rk_step(op, np.array([exact(t0)]), F_of, t0, dt, tol=1e-13, m_max=5)
    assert abs(u1[0] - exact(t0 + dt)) < 1e-13
    # the first stage alone is ETD1, exact for constant F
    want = math.exp(c * dt) * exact(t0) + (a + b * t0) * (math.exp(c * dt) - 1) / c
    assert abs(a1[0] - want) < 1e-13


def test_first_step_is_etd1():
    g = Grid((20, 20), (-2, -2), (2, 2))
    op = EBOperator(g, g.radius() - 1.3, 1.0)
    rng = np.random.default_rng(0)
    u0 = rng.uniform(0, 1, op.ncomp)
    F0 = u0 * (1 - u0)
    dt = 0.03
    got, _ = etd.etd2_step(op, u0, F0, F0, dt, exact=True)
    A = dt * op.C.toarray()
    want = u0 + dt * phi.combination_expm(A, [np.zeros_like(u0), F0 + op.C @ u0])
    assert np.max(np.abs(got - want)) < 1e-13


def _manufactured_error(n, R=1.0, box=1.6, scheme="etd2"):
    # u = e^{-t} cos(pi r / (2R)) on a fixed circle, u_t = Lap u + u(1-u) + s
    g = Grid((n, n), (-box, -box), (box, box))
    op = EBOperator(g, g.radius() - R, 1.0)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], axis=-1)
    r = np.sqrt(np.sum(X * X, axis=-1))
    k = math.pi / (2 * R)
    base = np.cos(k * r)
    lap = -k * k * np.cos(k * r) - k * np.sin(k * r) / np.where(r > 0, r, 1.0)
    lap = np.where(r > 0, lap, -2 * k * k)

    def F_of(u, t):
        ue = math.exp(-t) * base
        s = -ue - math.exp(-t) * lap - ue * (1 - ue)
        return u * (1 - u) + s

    dt = 0.5 * g.h
    T = 0.4
    nst = int(round(T / dt))
    dt = T / nst
    u = etd.run_fixed_domain(op, base.copy(), dt, nst, F_of, tol=1e-11, m_max=40, scheme=scheme)
    e = u - math.exp(-T) * base
    return np.max(np.abs(e)), math.sqrt(np.mean(e * e))


@pytest.mark.parametrize("scheme", ["etd2", "etd2rk"])
def test_manufactured_second_order(scheme):
    errs = [_manufactured_error(n, scheme=scheme) for n in (33, 65, 129)]
    for j in range(2):
        orders = [math.log2(errs[i][j] / errs[i + 1][j]) for i in range(2)]
        assert min(orders) > 1.6, (errs, orders)


def test_manufactured_etd1_first_order():
    # dt = h/2: the O(dt) time error dominates the O(h^2) space error
    errs = [_manufactured_error(n, scheme="etd1") for n in (33, 65, 129)]
    for j in range(2):
        orders = [math.log2(errs[i][j] / errs[i + 1][j]) for i in range(2)]
        assert all(0.8 < o < 1.4 for o in orders), (errs, orders)
    # ETD2 is more accurate at the same resolution
    assert _manufactured_error(65)[0] < errs[1][0]


def _peanut(n, tol=1e-10, scheme="etd2"):
    g = Grid((n, n), (-1.0, -1.0), (1.0, 1.0))
    x, y = g.coords()
    rho = 0.5 - np.exp(-20 * (x ** 2 + (y - 0.25) ** 2)) - np.exp(-20 * (x ** 2 + (y + 0.25) ** 2))

    def phi_fn(X):
        xx, yy = X[..., 0], X[..., 1]
        e1 = np.exp(-20 * (xx ** 2 + (yy - 0.25) ** 2))
        e2 = np.exp(-20 * (xx ** 2 + (yy + 0.25) ** 2))
        gx = 40 * xx * (e1 + e2)
        gy = 40 * (yy - 0.25) * e1 + 40 * (yy + 0.25) * e2
        return 0.5 - e1 - e2, np.stack([gx, gy], -1)

    beta = lambda X: 0.25 - X[..., 0] ** 2 - X[..., 1] ** 2
    op = EBOperator(g, rho, beta, phi_fn=phi_fn, boundary_data=True)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    r2 = np.sum(X ** 2, -1)

    def u_gamma(t):
        return lambda P: math.exp(-t) * (np.sum(P ** 2, -1) - 0.25)

    def F_of(u, t):
        # source of Sec. 4.2 for u = e^{-t}(r^2 - 1/4), beta = 1/4 - r^2: f = e^{-t}(28 r^2 - 3)/4
        return math.exp(-t) * (28 * r2 - 3) / 4 + op.boundary_rhs(u_gamma(t))

    dt = g.h
    nst = int(round(0.1 / dt))
    u = etd.run_fixed_domain(op, r2 - 0.25, dt, nst, F_of, tol=tol, m_max=40, scheme=scheme)
    e = u - math.exp(-nst * dt) * (r2 - 0.25)
    assert np.sum(op.kinds == 3) > 0  # the non-convex neck exercises case 3
    return np.max(np.abs(e)), math.sqrt(np.mean(e * e))


def _golden(path=GOLDEN):
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        n, s, li, l2 = line.split()
        rows.append((int(n), int(s), float(li), float(l2)))
    return rows


def test_table1_etd2_peanut():
    rows = [r for r in _golden() if r[0] <= 321]
    errs = [_peanut(n) for n, _, _, _ in rows]
    for (n, _, li, l2), (gi, g2) in zip(rows, errs):
        assert li / 3 <= gi <= 3 * li, (n, gi, li)
        assert l2 / 3 <= g2 <= 3 * l2, (n, g2, l2)
    # observed order from 81^2 to 321^2 (paper: about 2)
    assert math.log2(errs[0][0] / errs[-1][0]) / 2 > 1.5
    assert math.log2(errs[0][1] / errs[-1][1]) / 2 > 1.5


@pytest.mark.slow
def test_table1_etd2_peanut_641():
    n, _, li, l2 = [r for r in _golden() if r[0] == 641][0]
    gi, g2 = _peanut(n)
    assert li / 3 <= gi <= 3 * li and l2 / 3 <= g2 <= 3 * l2


def test_table1_etd2rk_peanut():
    rows = [r for r in _golden(GOLDEN_RK) if r[0] <= 321]
    errs = [_peanut(n, scheme="etd2rk") for n, _, _, _ in rows]
    for (n, _, li, l2), (gi, g2) in zip(rows, errs):
        assert li / 3 <= gi <= 3 * li, (n, gi, li)
        assert l2 / 3 <= g2 <= 3 * l2, (n, g2, l2)
    assert math.log2(errs[0][0] / errs[-1][0]) / 2 > 1.5
    assert math.log2(errs[0][1] / errs[-1][1]) / 2 > 1.5


@pytest.mark.slow
def test_table1_etd2rk_peanut_641():
    n, _, li, l2 = [r for r in _golden(GOLDEN_RK) if r[0] == 641][0]
    gi, g2 = _peanut(n, scheme="etd2rk")
    assert li / 3 <= gi <= 3 * li and l2 / 3 <= g2 <= 3 * l2


def _peanut_stability(n, dts, t_end=0.2, tol=1e-8):
    """l2 / l-inf errors and max |u| at t_end of ETD2 on the peanut problem
    (Sec. 4.2.1) for each time step of `dts`, and a lower bound of the
    spectral radius of -C (Rayleigh quotient after power iterations)."""
    g = Grid((n, n), (-1.0, -1.0), (1.0, 1.0))
    x, y = g.coords()
    rho = 0.5 - np.exp(-20 * (x ** 2 + (y - 0.25) ** 2)) - np.exp(-20 * (x ** 2 + (y + 0.25) ** 2))

    def phi_fn(X):
        xx, yy = X[..., 0], X[..., 1]
        e1 = np.exp(-20 * (xx ** 2 + (yy - 0.25) ** 2))
        e2 = np.exp(-20 * (xx ** 2 + (yy + 0.25) ** 2))
        return 0.5 - e1 - e2, np.stack([40 * xx * (e1 + e2), 40 * (yy - 0.25) * e1 + 40 * (yy + 0.25) * e2], -1)

    op = EBOperator(g, rho, lambda X: 0.25 - X[..., 0] ** 2 - X[..., 1] ** 2, phi_fn=phi_fn, boundary_data=True)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    r2 = np.sum(X ** 2, -1)

    def F_of(u, t):
        return math.exp(-t) * (28 * r2 - 3) / 4 + op.boundary_rhs(lambda P: math.exp(-t) * (np.sum(P ** 2, -1) - 0.25))

    v = np.random.default_rng(0).standard_normal(op.ncomp)
    for _ in range(60):
        v = -(op.C @ v)
        v /= np.linalg.norm(v)
    lam = float(v @ (-(op.C @ v)))
    out = []
    for dt in dts:
        nst = int(round(t_end / dt))
        u = etd.run_fixed_domain(op, r2 - 0.25, dt, nst, F_of, tol=tol, m_max=40)
        e = u - math.exp(-t_end) * (r2 - 0.25)
        out.append((math.sqrt(np.mean(e * e)), np.max(np.abs(e)), np.max(np.abs(u))))
    return out, lam, math.exp(-t_end) * np.max(np.abs(r2 - 0.25))


def _check_stability(dts, res, lam, umax):
    for dt, (l2, li, um) in zip(dts, res):
        # the explicit Euler / RK2 amplification of the stiffest mode exceeds
        # 1 at every step of the sweep: the problem is stiff there
        assert dt * lam > 2.0, (dt, lam)
        # ETD2 stays bounded: error below 1% of max |u|, no growth of u
        assert l2 <= 1e-2 * umax and li <= 2e-2 * umax, (dt, l2, li)
        assert um <= 1.05 * umax, (dt, um)
    # the error does not grow as dt shrinks (down to the spatial error)
    for a, b in zip(res[:-1], res[1:]):
        assert b[0] <= 1.05 * a[0]


def test_stability_etd2_peanut():
    """Stability (Sec. 4.2.2, Fig. 5): ETD2 on the peanut problem to t = 0.2
    stays bounded for steps up to dt = 0.1, far beyond the explicit limit
    2 / rho(C).  On h = 0.008 (251^2) here; h = 0.004 as printed is the slow
    test below."""
    dts = [0.1, 1e-2, 1e-3]
    res, lam, umax = _peanut_stability(251, dts)
    _check_stability(dts, res, lam, umax)


@pytest.mark.slow
def test_stability_etd2_peanut_h004():
    """As above at the paper's h = 0.004 (501^2) with dt = 0.1 ... 1e-4."""
    dts = [0.1, 1e-2, 1e-3, 1e-4]
    res, lam, umax = _peanut_stability(501, dts)
    _check_stability(dts, res, lam, umax)


# ---- ETD3RK / ETD4RK (Sec. 3.2)

def _poly_forced_exact(c, coef, t0, u0, dt):
    """u(t0 + dt) for u' = c u + q(t), q a polynomial (coefficients low to
    high), by variation of constants with scipy's adaptive quadrature."""
    from scipy.integrate import quad

    q = lambda t: sum(a * t ** k for k, a in enumerate(coef))
    val = quad(lambda s: math.exp(c * (dt - s)) * q(t0 + s), 0.0, dt, epsabs=1e-16, epsrel=1e-15)[0]
    return math.exp(c * dt) * u0 + val


@pytest.mark.parametrize("step", [etd.etd3rk_step, etd.etd4rk_step])
def test_etdrk34_exact_for_quadratic_forcing(step):
    # With F independent of U the final stage integrates the quadratic
    # interpolant of F through t_n, t_n + dt/2, t_n + dt exactly, so a forcing
    # quadratic in t is reproduced to rounding.  The phi_3 term carries the
    # t^2 part: a phi_3 normalised the standard way instead of by Eq. 3.7
    # fails here.
    c, coef, t0, dt, u0 = -3.0, (0.7, -1.3, 0.9), 0.3, 0.2, 0.4
    op = _ScalarOp(c)
    F_of = lambda u, t: np.full_like(u, coef[0] + coef[1] * t + coef[2] * t * t)
    u1 = step(op, np.array([u0]), F_of, t0, dt, tol=1e-14, m_max=8)[0]
    assert abs(u1[0] - _poly_forced_exact(c, coef, t0, u0, dt)) < 1e-14
    # a cubic forcing is not integrated exactly (the interpolant is quadratic)
    Fc = lambda u, t: np.full_like(u, t ** 3)
    u3 = step(op, np.array([u0]), Fc, t0, dt, tol=1e-14, m_max=8)[0]
    assert abs(u3[0] - _poly_forced_exact(c, (0.0, 0.0, 0.0, 1.0), t0, u0, dt)) > 1e-8


@pytest.mark.parametrize("step", [etd.etd3rk_step, etd.etd4rk_step])
def test_etdrk34_linear_is_expm(step):
    # F = 0: every stage is phi_0 alone and U_{n+1} = exp(dt C) U_n (scipy's expm)
    import scipy.linalg as sl

    g = Grid((14, 14), (-2, -2), (2, 2))
    op = EBOperator(g, g.radius() - 1.3, 1.0)
    u0 = np.random.default_rng(2).uniform(-1, 1, op.ncomp)
    dt = 0.05
    u1 = step(op, u0, lambda u, t: np.zeros_like(u), 0.0, dt, tol=1e-13, m_max=40)[0]
    want = sl.expm(dt * op.C.toarray()) @ u0
    assert np.max(np.abs(u1 - want)) <= 1e-11 * np.max(np.abs(want))


def test_etdrk34_scalar_orders():
    # u' = c u + u (1 - u) = r u - u^2 (r = 1 + c), a Bernoulli equation with
    # the closed form u = r u0 e^{rt} / (r + u0 (e^{rt} - 1)).
    c, u0, T = -2.0, 0.6, 1.0
    r = 1.0 + c
    exact = r * u0 * math.exp(r * T) / (r + u0 * (math.exp(r * T) - 1.0))
    op = _ScalarOp(c)
    F_of = lambda u, t: u * (1.0 - u)
    for step, order in ((etd.etd3rk_step, 3), (etd.etd4rk_step, 4)):
        errs = []
        for n in (10, 20, 40, 80):
            u, t = np.array([u0]), 0.0
            for _ in range(n):
                u = step(op, u, F_of, t, T / n, tol=1e-14, m_max=8)[0]
                t += T / n
            errs.append(abs(u[0] - exact))
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(1, 3)]
        assert min(orders) > order - 0.4, (errs, orders)


def test_etdrk34_stiff_system_orders():
    # The EB system of a small disc with the logistic reaction (spectral
    # radius of C about 108): temporal convergence against scipy's DOP853 at
    # tight tolerance, the combinations by the dense augmented expm.  ETD4RK
    # reaches order 4 and ETD3RK approaches 3, far below ETD2RK's error.
    from scipy.integrate import solve_ivp

    g = Grid((16, 16), (-2, -2), (2, 2))
    op = EBOperator(g, g.radius() - 1.3, 1.0)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    u0 = 0.5 + 0.4 * np.cos(X[:, 0]) * np.sin(X[:, 1] + 0.3)
    F_of = lambda u, t: u * (1.0 - u)
    C = op.C.toarray()
    T = 0.8
    ref = solve_ivp(lambda t, u: C @ u + F_of(u, t), (0.0, T), u0, method="DOP853", rtol=3e-14,
                    atol=1e-15).y[:, -1]

    def err(scheme, n):
        u = etd.run_fixed_domain(op, u0, T / n, n, F_of, exact=True, scheme=scheme)
        return np.max(np.abs(u - ref))

    e4 = [err("etd4rk", n) for n in (32, 64, 128)]
    assert min(math.log2(e4[i] / e4[i + 1]) for i in range(2)) > 3.5, e4
    e3 = [err("etd3rk", n) for n in (128, 256, 512)]
    assert math.log2(e3[1] / e3[2]) > 2.6, e3
    e2 = err("etd2rk", 64)
    assert e4[1] < 5e-3 * e2 and err("etd3rk", 64) < 5e-3 * e2


# ---- multistep ETD3 (Eq. 3.8b, s = 3)

def _g_m(m, z):
    """g_m(z) of Eq. 3.8b by quadrature: (-1)^m int_0^1 e^{(1-l) z} binom(-l, m) dl."""
    from scipy.integrate import quad

    def binom(x, k):
        out = 1.0
        for i in range(k):
            out *= (x - i) / (i + 1)
        return out

    return (-1) ** m * quad(lambda l: math.exp((1.0 - l) * z) * binom(-l, m), 0.0, 1.0, epsabs=1e-15,
                            epsrel=1e-14)[0]


def test_etd3_multistep_matches_eq38b():
    # one scalar step from the vectors against Eq. 3.8b written out with the
    # quadrature weights and the backward differences of F
    for c, dt in ((-3.0, 0.2), (-40.0, 0.05), (0.5, 0.1)):
        op = _ScalarOp(c)
        u, F0, F1, F2 = 0.4, 0.7, -0.2, 1.1  # F_n, F_{n-1}, F_{n-2}
        z = c * dt
        d1, d2 = F0 - F1, F0 - 2 * F1 + F2
        want = math.exp(z) * u + dt * (_g_m(0, z) * F0 + _g_m(1, z) * d1 + _g_m(2, z) * d2)
        got = etd.etd3_step(op, np.array([u]), np.array([F0]), np.array([F1]), np.array([F2]), dt, tol=1e-14,
                            m_max=8)[0][0]
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (c, got, want)


def test_etd3_multistep_exact_for_quadratic_forcing():
    # with exact history the step integrates the quadratic through
    # t_{n-2}, t_{n-1}, t_n, so a forcing quadratic in t is exact
    c, coef, t0, dt, u0 = -3.0, (0.7, -1.3, 0.9), 0.3, 0.2, 0.4
    op = _ScalarOp(c)
    q = lambda t: coef[0] + coef[1] * t + coef[2] * t * t
    got = etd.etd3_step(op, np.array([u0]), np.array([q(t0)]), np.array([q(t0 - dt)]), np.array([q(t0 - 2 * dt)]),
                        dt, tol=1e-14, m_max=8)[0][0]
    assert abs(got - _poly_forced_exact(c, coef, t0, u0, dt)) < 1e-14
    # ETD2 with the same data is not exact (its interpolant is linear)
    e2 = etd.etd2_step(op, np.array([u0]), np.array([q(t0)]), np.array([q(t0 - dt)]), dt, tol=1e-14, m_max=8)[0][0]
    assert abs(e2 - _poly_forced_exact(c, coef, t0, u0, dt)) > 1e-6


def test_etd3_multistep_order_3():
    # the Bernoulli equation u' = c u + u (1 - u), started from the closed form
    # at t_0, t_1, t_2 (exact history), then multistep ETD3 steps to T
    c, u0, T = -2.0, 0.6, 1.0
    r = 1.0 + c
    exact = lambda t: r * u0 * math.exp(r * t) / (r + u0 * (math.exp(r * t) - 1.0))
    op = _ScalarOp(c)
    F = lambda u: u * (1.0 - u)
    errs = []
    for n in (10, 20, 40, 80):
        dt = T / n
        us = [exact(0.0), exact(dt), exact(2 * dt)]
        for k in range(2, n):
            Fs = [F(np.array([us[k - i]])) for i in range(3)]
            us.append(etd.etd3_step(op, np.array([us[k]]), Fs[0], Fs[1], Fs[2], dt, tol=1e-14, m_max=8)[0][0])
        errs.append(abs(us[n] - exact(T)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(1, 3)]
    assert min(orders) > 2.7, (errs, orders)


def test_etd3_multistep_start_up_reading():
    # with no earlier F the first step is ETD1, with one it is ETD2
    g = Grid((14, 14), (-2, -2), (2, 2))
    op = EBOperator(g, g.radius() - 1.3, 1.0)
    u0 = np.random.default_rng(6).uniform(0, 1, op.ncomp)
    F_of = lambda u, t: u * (1.0 - u)
    dt = 0.05
    u1 = etd.run_fixed_domain(op, u0, dt, 1, F_of, tol=1e-12, scheme="etd3")
    assert np.max(np.abs(u1 - etd.etd1_step(op, u0, F_of(u0, 0), dt, tol=1e-12)[0])) <= 1e-14
    u2 = etd.run_fixed_domain(op, u0, dt, 2, F_of, tol=1e-12, scheme="etd3")
    want = etd.etd2_step(op, u1, F_of(u1, dt), F_of(u0, 0), dt, tol=1e-12)[0]
    assert np.max(np.abs(u2 - want)) <= 1e-14
