"""Pins for oracle.eb: classification by brute force, the case-2 weight by the
paper's Lagrange formula written pointwise, case 3 against barycentric
coordinates, structural properties (symmetry, sign pattern, spectrum), the
3D hyperplane rule reducing to the 2D rule, and second-order convergence of
the Poisson solve (Sec. 4.1's exact solution and beta, on a disc)."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import eb
from oracle.grid import Grid


def _disc(n, R=1.3, box=2.0, center=(0.0, 0.0)):
    g = Grid((n, n), (-box, -box), (box, box))
    x, y = g.coords()
    return g, np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2) - R


def _peanut_phi(x, y):
    return 0.5 - np.exp(-20 * (x ** 2 + (y - 0.25) ** 2)) - np.exp(-20 * (x ** 2 + (y + 0.25) ** 2))


def test_classify_brute_force():
    g = Grid((23, 23), (-1.1, -1.1), (1.1, 1.1))
    x, y = g.coords()
    ph = _peanut_phi(x, y)
    inside, ghost, comp = eb.classify(g, ph)
    for i in range(23):
        for j in range(23):
            ins = ph[i, j] < 0
            nbs = []
            for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                a, b = i + di, j + dj
                nbs.append(0 <= a < 23 and 0 <= b < 23 and ph[a, b] < 0)
            assert inside[i, j] == ins
            assert comp[i, j] == (ins and all(nbs))
            assert ghost[i, j] == (ins and not all(nbs))


def test_domain_margin_error():
    g, ph = _disc(16, R=1.9, box=2.0)
    with pytest.raises(eb.DomainError):
        eb.classify(g, ph)


@pytest.mark.parametrize("ndim", [2, 3, 4])
def test_structure_symmetric_mmatrix_spectrum(ndim):
    n = {2: 26, 3: 16, 4: 13}[ndim]
    g = Grid((n,) * ndim, (-2.0,) * ndim, (2.0,) * ndim)
    x = g.coords()
    a = [1.0, 0.8, 0.9, 0.7][:ndim]
    ph = np.sqrt(sum((x[d] / a[d]) ** 2 for d in range(ndim))) - 1.0
    rng = np.random.default_rng(ndim)
    beta = 1.0 + 0.3 * rng.uniform(-1, 1, size=g.n)
    op = eb.EBOperator(g, ph, beta)
    C = op.C.toarray()
    assert op.ncomp > 10
    assert np.array_equal(C, C.T)  # bitwise symmetric
    off = C - np.diag(np.diag(C))
    assert np.all(off >= 0.0)
    assert np.all(np.diag(C) < 0.0)
    assert np.all(-np.diag(C) >= off.sum(axis=1) * (1.0 - 1e-14))  # diagonal dominance (M-matrix)
    lam = np.linalg.eigvalsh(C)
    assert lam.max() < 0.0
    assert lam.min() >= -4.0 * ndim * beta.max() / g.h ** 2
    assert set(np.unique(op.kinds)) <= {1, 2, 3}


def test_case2_weight_is_lagrange_formula():
    g, ph = _disc(30, R=1.37)
    op = eb.EBOperator(g, ph, 1.0)
    st = eb.strides(g.n)
    pf = ph.ravel()
    n2 = 0
    for row, p in enumerate(op.index):
        for d in range(2):
            for si, s in enumerate((-1, 1)):
                if op.kinds[row, 2 * d + si] != 2:
                    continue
                n2 += 1
                q = p + s * st[d]
                r = q + s * st[d]
                # coordinate along the grid line, measured from p in units of h
                yp, yq = 0.0, 1.0
                # secant: linear interpolation of phi between q and r vanishes at yG
                yG = yq + pf[q] / (pf[q] - pf[r])
                # Eq. DirichletLineByLine: u_GP = u_G (y_GP - y_p)/(y_G - y_p) - u_p (y_GP - y_G)/(y_G - y_p)
                g1 = -(yq - yG) / (yG - yp)
                gG = (yq - yp) / (yG - yp)
                assert abs(op.weights[row, 2 * d + si] - g1) < 1e-14
                assert 0.0 < g1 <= 0.5 + 1e-15 and 0.5 <= gG <= 1.0  # |g| <= 1 (Sec. 2)
    assert n2 > 20


def test_rbf_equals_barycentric():
    rng = np.random.default_rng(5)
    h = 0.05
    for _ in range(50):
        xp, xq, g1, g2 = (rng.uniform(-1, 1, 2) for _ in range(4))
        c = eb.rbf_weights_2d(xp, xq, g1, g2, h)
        T = np.array([[1.0, 1.0, 1.0], [xp[0], g1[0], g2[0]], [xp[1], g1[1], g2[1]]])
        lam = np.linalg.solve(T, np.array([1.0, xq[0], xq[1]]))
        assert np.allclose(c, lam, atol=1e-9 * max(1.0, np.abs(lam).max()))
        # affine data reproduced exactly
        f = lambda z: 0.3 - 1.7 * z[0] + 2.2 * z[1]
        assert abs(c[0] * f(xp) + c[1] * f(g1) + c[2] * f(g2) - f(xq)) < 1e-9


def test_case3_hyperplane_reduces_to_2d():
    # A long cylinder in 3D: away from its caps, the x/y ghost faces see the
    # same geometry as the disc cross-section, and the N >= 3 hyperplane rule
    # must give the 2D (RBF / barycentric) weights.
    n2 = 34
    R = 1.23
    g2, ph2 = _disc(n2, R=R, box=2.0, center=(0.031, -0.017))
    op2 = eb.EBOperator(g2, ph2, 1.0)
    # equal spacing on z as well: h = 4/33, 20 nodes
    g3 = Grid((n2, n2, 20), (-2.0, -2.0, -1.0 * 19 * (4.0 / 33) / 2), (2.0, 2.0, 1.0 * 19 * (4.0 / 33) / 2))
    x, y, z = g3.coords()
    cyl = np.sqrt((x - 0.031) ** 2 + (y + 0.017) ** 2) - R
    cap = np.abs(z) - 0.5 * 19 * (4.0 / 33) + 3.5 * g3.h
    ph3 = np.maximum(cyl, cap)
    op3 = eb.EBOperator(g3, ph3, 1.0)
    k_mid = 10
    w2 = {}
    for row, p in enumerate(op2.index):
        i, j = np.unravel_index(p, g2.n)
        w2[(i, j)] = (op2.kinds[row], op2.weights[row])
    ncase3 = 0
    for row, p in enumerate(op3.index):
        i, j, k = np.unravel_index(p, g3.n)
        if k != k_mid:
            continue
        kinds2, wts2 = w2[(i, j)]
        assert np.array_equal(op3.kinds[row, :4], kinds2)
        assert np.allclose(op3.weights[row, :4], wts2, atol=1e-10)
        ncase3 += int(np.sum(kinds2 == 3))
    assert ncase3 > 0


def _poisson_error(n):
    # Sec. 4.1: u = e^x (x^2 sin y + y^2), beta = 2 + sin(x y); here on a disc of
    # radius 0.6 in [-1,1]^2 with the exact u as Dirichlet data.
    g = Grid((n, n), (-1.0, -1.0), (1.0, 1.0))
    x, y = g.coords()
    ph = np.sqrt(x * x + y * y) - 0.6

    def u_ex(X):
        return np.exp(X[..., 0]) * (X[..., 0] ** 2 * np.sin(X[..., 1]) + X[..., 1] ** 2)

    def beta(X):
        return 2.0 + np.sin(X[..., 0] * X[..., 1])

    def phi_fn(X):
        r = np.sqrt(np.sum(X * X, axis=-1))
        return r - 0.6, X / r[:, None]

    op = eb.EBOperator(g, ph, beta, phi_fn=phi_fn, boundary_data=True)
    X = np.stack([c.ravel()[op.index] for c in g.coords()], axis=-1)
    xx, yy = X[:, 0], X[:, 1]
    # f = div(beta grad u), derived by hand:
    e = np.exp(xx)
    ux = e * (xx ** 2 * np.sin(yy) + yy ** 2) + e * 2 * xx * np.sin(yy)
    uy = e * (xx ** 2 * np.cos(yy) + 2 * yy)
    uxx = e * (xx ** 2 * np.sin(yy) + yy ** 2) + 2 * e * 2 * xx * np.sin(yy) + e * 2 * np.sin(yy)
    uyy = e * (-xx ** 2 * np.sin(yy) + 2)
    b = 2.0 + np.sin(xx * yy)
    bx, by = yy * np.cos(xx * yy), xx * np.cos(xx * yy)
    f = b * (uxx + uyy) + bx * ux + by * uy
    rhs = f - op.boundary_rhs(u_ex)
    u = spla.spsolve(op.C.tocsc(), rhs)
    return np.max(np.abs(u - u_ex(X)))


def test_poisson_second_order():
    errs = [_poisson_error(n) for n in (41, 81, 161)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-3
    assert min(orders) > 1.6, (errs, orders)
