"""Pins for oracle.phi: scalar phi_k against the integral definition (Eq. 3.7)
and arbitrary-precision closed forms, the two exact combination routes
against each other and against an ODE solve of Eq. 3.10."""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle import phi

mpmath = pytest.importorskip("mpmath")


def phi_mp(k, z):
    """phi_k(z) = (e^z - sum_{j<k} z^j/j!) / z^k in 60-digit arithmetic."""
    mpmath.mp.dps = 60
    z = mpmath.mpf(z)
    if z == 0:
        return 1.0 / math.factorial(k)
    s = mpmath.e ** z - sum(z ** j / mpmath.factorial(j) for j in range(k))
    return float(s / z ** k)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_phi_scalar_closed_form(k):
    zs = np.array([-40.0, -7.5, -1.0, -0.999, -0.3, -1e-6, 0.0, 1e-6, 0.2, 0.999, 1.0, 3.0])
    got = phi.phi_scalar(k, zs)
    want = np.array([phi_mp(k, z) for z in zs])
    assert np.allclose(got, want, rtol=2e-13, atol=0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_phi_scalar_integral_definition(k):
    # Eq. 3.7 with the (k-1)! of the standard normalisation:
    # phi_k(z) = int_0^1 e^{(1-l) z} l^{k-1} / (k-1)! dl
    for z in (-12.0, -2.0, -0.5, 0.0, 0.7):
        val, _ = quad(lambda l: math.exp((1 - l) * z) * l ** (k - 1) / math.factorial(k - 1), 0.0, 1.0,
                      epsabs=0, epsrel=1e-13)
        assert abs(phi.phi_scalar(k, np.array([z]))[0] - val) <= 5e-13 * abs(val)


def test_paper_recursion_k_le_2():
    # Eq. 3.8 (paper normalisation) phi_{k+1} = (k phi_k - 1)/z agrees with the
    # standard one for k <= 2: phi_2 = (phi_1 - 1)/z.
    z = np.array([-5.0, -1.5, 2.0])
    assert np.allclose(phi.phi_scalar(2, z), (1 * phi.phi_scalar(1, z) - 1.0) / z, rtol=1e-14)


def test_paper_phi3_is_twice_standard():
    # The phi_3 of the ETD3RK / ETD4RK formulas: Eq. 3.7 (the integral of
    # e^{(1-l) z} l^2 over [0, 1], by quadrature) and Eq. 3.8 with k = 2,
    # (2 phi_2 - 1) / z, both equal twice the standard phi_3.
    for z in (-6.0, -1.5, -0.1, 0.7):
        eq37 = quad(lambda l: math.exp((1.0 - l) * z) * l * l, 0.0, 1.0, epsabs=1e-15, epsrel=1e-14)[0]
        eq38 = (2.0 * phi.phi_scalar(2, np.array([z]))[0] - 1.0) / z
        std3 = phi.phi_scalar(3, np.array([z]))[0]
        assert abs(eq37 - 2.0 * std3) <= 1e-13 * abs(eq37)
        assert abs(eq38 - 2.0 * std3) <= 1e-12 * abs(eq38)


def _spd_neg(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = -np.linspace(0.05, 9.0, n)
    return (Q * lam) @ Q.T

@pytest.mark.parametrize("p", [1, 2, 3])
def test_combination_expm_vs_eig(p):
    A = _spd_neg(30, p)
    rng = np.random.default_rng(10 + p)
    vs = [rng.standard_normal(30) for _ in range(p + 1)]
    a = phi.combination_expm(A, vs)
    b = phi.combination_eig(A, vs)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))

def test_combination_scalar_matrix():
    # 1 x 1 A = [z]: sum phi_k(z) v_k in closed form
    for z in (-3.0, -0.25, 0.5):
        vs = [np.array([1.3]), np.array([-0.7]), np.array([2.1])]
        want = sum(phi_mp(k, z) * vs[k][0] for k in range(3))
        assert abs(phi.combination_expm(np.array([[z]]), vs)[0] - want) < 1e-13 * abs(want)

@pytest.mark.parametrize("p", [2, 3])
def test_combination_is_ode_solution(p):
    # Eq. 3.10: y' = A y + sum_{k=1}^p t^{k-1}/(k-1)! v_k, y(0) = v_0, y(1) is the sum.
    A = _spd_neg(8, 7)
    rng = np.random.default_rng(3)
    vs = [rng.standard_normal(8) for _ in range(p + 1)]

    def f(t, y):
        return A @ y + sum(t ** (k - 1) / math.factorial(k - 1) * vs[k] for k in range(1, p + 1))
    sol = solve_ivp(f, (0.0, 1.0), vs[0], method="DOP853", rtol=1e-13, atol=1e-14)
    assert np.max(np.abs(sol.y[:, -1] - phi.combination_expm(A, vs))) < 1e-10

def test_phi_columns_diagonal_and_triangular():
    # diagonal H: phi_k(H) e1 = phi_k(h11) e1
    H = np.diag([-2.0, -0.5, -4.0])
    cols = phi.phi_columns_expm(H, 3)
    for k in range(1, 4):
        assert abs(cols[0, k - 1] - phi_mp(k, -2.0)) < 1e-14
        assert np.all(cols[1:, k - 1] == 0.0)
    # lower triangular 2 x 2 [[a, 0], [b, c]]: f(H) e1 = (f(a), b (f(a) - f(c)) / (a - c))
    a, b, c = -1.2, 0.8, -3.1
    cols = phi.phi_columns_expm(np.array([[a, 0.0], [b, c]]), 3)
    for k in range(1, 4):
        fa, fc = phi_mp(k, a), phi_mp(k, c)
        assert abs(cols[0, k - 1] - fa) < 1e-14
        assert abs(cols[1, k - 1] - b * (fa - fc) / (a - c)) < 1e-13
