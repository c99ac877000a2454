"""Pins for oracle.adjoint: the adjoint gradients of a terminal loss through
ETD2 steps equal central finite differences of the forward trajectory
(exact phi-functions by dense expm), for u_0, the node field beta (at
computational and ghost nodes) and alpha; the time quadrature of the beta
term converges."""
import numpy as np
import pytest

from oracle import adjoint
from oracle.eb import EBOperator
from oracle.grid import Grid


def _setup(ndim, n, R, seed):
    g = Grid((n,) * ndim, (-1.5,) * ndim, (1.5,) * ndim)
    x = g.coords()
    r = np.sqrt(sum(c * c for c in x))
    ph = r - R
    beta = 1.0 + 0.3 * np.sin(1.7 * x[0] + 0.4) * np.cos(1.1 * x[1])
    rng = np.random.default_rng(seed)
    return g, ph, beta, rng


def _loss(g, ph, beta, u0, dt, nsteps, alpha, K, target):
    op = EBOperator(g, ph, beta)
    pe = adjoint.PhiEval(op, exact=True)
    us = adjoint.forward(op, u0, dt, nsteps, alpha, K, pe)
    r = us[-1] - target
    return 0.5 * float(np.dot(r, r))


@pytest.mark.parametrize("ndim,n,R", [(2, 14, 1.0), (3, 12, 0.8)])
def test_adjoint_matches_finite_differences(ndim, n, R):
    g, ph, beta, rng = _setup(ndim, n, R, ndim)
    op = EBOperator(g, ph, beta)
    assert op.ncomp > 5 and np.any(op.kinds >= 2)
    u0 = rng.uniform(0.2, 0.9, op.ncomp)
    target = rng.uniform(0.0, 0.5, op.ncomp)
    dt, nsteps, alpha, K = 0.05, 3, 1.0, 1.0
    pe = adjoint.PhiEval(op, exact=True)
    L, gu, gb, ga = adjoint.trajectory_gradient(op, u0, dt, nsteps, alpha, K, target, pe, nquad=10)
    eps = 1e-6

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b), 1e-8)

    # u_0
    for i in rng.choice(op.ncomp, 4, replace=False):
        up, um = u0.copy(), u0.copy()
        up[i] += eps
        um[i] -= eps
        fd = (_loss(g, ph, beta, up, dt, nsteps, alpha, K, target) -
              _loss(g, ph, beta, um, dt, nsteps, alpha, K, target)) / (2 * eps)
        assert close(gu[i], fd), (i, gu[i], fd)
    # alpha
    fd = (_loss(g, ph, beta, u0, dt, nsteps, alpha + eps, K, target) -
          _loss(g, ph, beta, u0, dt, nsteps, alpha - eps, K, target)) / (2 * eps)
    assert close(ga, fd), (ga, fd)
    # beta at two computational nodes and two ghost nodes
    comp_nodes = np.flatnonzero(op.comp.ravel())
    ghost_nodes = np.flatnonzero(op.ghost.ravel())
    picks = list(rng.choice(comp_nodes, 2, replace=False)) + list(rng.choice(ghost_nodes, 2, replace=False))
    for fl in picks:
        bp, bm = beta.copy().ravel(), beta.copy().ravel()
        bp[fl] += eps
        bm[fl] -= eps
        fd = (_loss(g, ph, bp.reshape(g.n), u0, dt, nsteps, alpha, K, target) -
              _loss(g, ph, bm.reshape(g.n), u0, dt, nsteps, alpha, K, target)) / (2 * eps)
        assert close(gb.ravel()[fl], fd), (fl, gb.ravel()[fl], fd)


def test_beta_quadrature_converges():
    g, ph, beta, rng = _setup(2, 14, 1.0, 5)
    op = EBOperator(g, ph, beta)
    pe = adjoint.PhiEval(op, exact=True)
    u_n = rng.uniform(0.2, 0.9, op.ncomp)
    lam = rng.standard_normal(op.ncomp)
    dt = 0.05  # |dt C| about 9, the stiffness of the workloads
    gbs = [adjoint.adjoint_step(op, pe, dt, u_n, u_n, lam, 1.0, 1.0, nq)[3] for nq in (4, 8, 16)]
    d1 = np.max(np.abs(gbs[1] - gbs[0]))
    d2 = np.max(np.abs(gbs[2] - gbs[1]))
    assert d2 < 1e-9 * np.max(np.abs(gbs[2])) and d2 < d1
