"""Pins for oracle.krylov: the adaptive Krylov phi-combination against the
dense augmented-matrix expm (oracle.phi, itself pinned against
eigendecomposition and closed forms), on EB operators in 2D/3D/4D, with
substepping, rejections and happy breakdown exercised."""
import numpy as np
import pytest

from oracle import krylov, phi
from oracle.eb import EBOperator
from oracle.grid import Grid


def _ball_op(ndim, n, R, beta=1.0):
    g = Grid((n,) * ndim, (-2.0,) * ndim, (2.0,) * ndim)
    x = g.coords()
    ph = np.sqrt(sum(c * c for c in x)) - R
    return EBOperator(g, ph, beta)


@pytest.mark.parametrize("ndim,n,R,dt,p", [(2, 30, 1.4, 0.02, 2), (3, 14, 1.3, 0.05, 2), (4, 13, 1.3, 0.1, 2),
                                           (2, 26, 1.2, 0.05, 1), (3, 14, 1.3, 0.02, 3)])
def test_phipm_matches_dense(ndim, n, R, dt, p):
    op = _ball_op(ndim, n, R)
    A = dt * op.C.toarray()
    rng = np.random.default_rng(ndim * 10 + p)
    vs = [rng.standard_normal(op.ncomp) for _ in range(p + 1)]
    exact = phi.combination_expm(A, vs)
    tol = 1e-9
    y, trace = krylov.phipm(lambda x: A @ x, vs, tol, 40, np.max(np.abs(A).sum(axis=1)))
    assert np.linalg.norm(y - exact) <= 20 * tol * np.linalg.norm(exact)
    assert abs(sum(t for t, _, _ in trace) - 1.0) < 1e-14


def test_phipm_substeps_and_rejections():
    # stiff operator and a small basis: forces tau < 1 and rejections
    op = _ball_op(2, 40, 1.6)
    dt = 0.5
    A = dt * op.C.toarray()
    rng = np.random.default_rng(1)
    vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
    exact = phi.combination_expm(A, vs)
    y, trace = krylov.phipm(lambda x: A @ x, vs, 1e-8, 10, np.max(np.abs(A).sum(axis=1)))
    assert len(trace) > 3
    assert any(r > 0 for _, _, r in trace)
    assert np.linalg.norm(y - exact) <= 1e-6 * np.linalg.norm(exact)


def test_phipm_happy_breakdown():
    # v's in a 2-dimensional invariant subspace: the basis breaks down at m = 2
    # and the result is exact.
    n = 50
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = -np.linspace(0.1, 5.0, n)
    A = (Q * lam) @ Q.T
    vs = [Q[:, 3] * 0.7 - Q[:, 9] * 0.2, Q[:, 3] * 1.1, Q[:, 9] * 0.4]
    exact = phi.combination_eig(A, vs)
    y, trace = krylov.phipm(lambda x: A @ x, vs, 1e-12, 30, np.max(np.abs(A).sum(axis=1)))
    assert trace[0][1] <= 2
    assert np.linalg.norm(y - exact) <= 1e-12 * np.linalg.norm(exact)


def test_phipm_zero_forcing():
    A = -np.eye(5)
    vs = [np.zeros(5), np.zeros(5), np.zeros(5)]
    y, trace = krylov.phipm(lambda x: A @ x, vs, 1e-8, 10, 1.0)
    assert np.all(y == 0.0)


def test_forced_trace_replay_is_identical():
    op = _ball_op(3, 14, 1.3)
    A = 0.2 * op.C.toarray()
    rng = np.random.default_rng(4)
    vs = [rng.standard_normal(op.ncomp) for _ in range(3)]
    y1, tr1 = krylov.phipm(lambda x: A @ x, vs, 1e-8, 20, np.max(np.abs(A).sum(axis=1)))
    y2, tr2 = krylov.phipm(lambda x: A @ x, vs, 1e-8, 20, np.max(np.abs(A).sum(axis=1)), forced_trace=tr1)
    assert np.array_equal(y1, y2)
    assert [t[:2] for t in tr1] == [t[:2] for t in tr2]
