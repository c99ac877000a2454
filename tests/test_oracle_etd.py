"""Pins for oracle.etd: ETD2 and ETD2RK on a scalar ODE in closed form,
first-order (ETD1) and second-order (ETD2, ETD2RK) convergence for a
manufactured solution on a fixed circle, and the paper's Table 1 (ETD2 and
ETD2RK on the peanut domain, Sec. 4.2.1) within a factor of 3."""
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
