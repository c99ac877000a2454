"""Pins for oracle.poisson on the virus-shaped domain of Sec. 4.1: the source
formula against symbolic differentiation, second-order convergence of the
solution in l2 and l-infinity (the order the paper reports, Sec. 4.1 and its
error figure), and the exact solution of a problem whose solution is affine
(the ghost-value interpolants reproduce affine data)."""
import math

import numpy as np
import pytest

from oracle import poisson
from oracle.eb import EBOperator
from oracle.grid import Grid
from paper_2209_15095_gb300 import inputs


def _virus_error(N):
    w = inputs.virus2d(N)
    g = Grid(w.n, w.lo, w.hi)
    op = EBOperator(g, w.phi0[0], w.beta_field, boundary_data=True)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    u = poisson.solve(op, op.from_grid(w.source), lambda P: inputs.virus_exact(P[..., 0], P[..., 1]))
    e = u - inputs.virus_exact(X[:, 0], X[:, 1])
    return np.max(np.abs(e)), math.sqrt(np.mean(e * e)), op


def test_virus_source_formula():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    u = sympy.exp(x) * (x ** 2 * sympy.sin(y) + y ** 2)
    beta = 2 + sympy.sin(x * y)
    f = sympy.diff(beta * sympy.diff(u, x), x) + sympy.diff(beta * sympy.diff(u, y), y)
    fn = sympy.lambdify((x, y), f, "numpy")
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, (200, 2))
    assert np.max(np.abs(fn(P[:, 0], P[:, 1]) - inputs.virus_source(P[:, 0], P[:, 1]))) < 1e-12


def test_virus_second_order():
    errs = [_virus_error(N)[:2] for N in (50, 100, 200)]
    for j in range(2):
        orders = [math.log2(errs[i][j] / errs[i + 1][j]) for i in range(2)]
        assert min(orders) > 1.6, (errs, orders)


def test_affine_solution_exact():
    # u = 1 + 2x - 3y solves div(grad u) = 0; unclamped ghost values
    # interpolate affine data exactly (cases 2 and 3), so the discrete solution
    # is exact.  At N = 200 no ghost weight of this domain is clamped.
    w = inputs.virus2d(200)
    g = Grid(w.n, w.lo, w.hi)
    op = EBOperator(g, w.phi0[0], 1.0, boundary_data=True)
    assert np.sum(op.kinds == 3) > 0 and op.nclamp == 0
    X = np.stack([c.ravel()[op.index] for c in g.coords()], -1)
    ua = lambda P: 1.0 + 2.0 * P[..., 0] - 3.0 * P[..., 1]
    u = poisson.solve(op, np.zeros(op.ncomp), ua)
    assert np.max(np.abs(u - ua(X))) < 1e-11
