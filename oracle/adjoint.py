"""Adjoint of the ETD2 step on a frozen domain (gradients of a terminal loss
with respect to u_0, the node field beta and the reaction rate alpha).

Forward (Sec. 3.1, ETD2; F_{-1} = F_0):
    u_{n+1} = phi_0(A) u_n + dt phi_1(A) F(u_n) + dt phi_2(A) (F(u_n) - F(u_{n-1})),
    A = dt C(beta),  F(u) = alpha u (1 - u / K).
C is symmetric (Sec. 2: the ghost rows only change the diagonal), so
phi_k(A)^T = phi_k(A).  With lambda = dL/du_{n+1} and Phi_k = phi_k(A) lambda:
    dL/du_n     += Phi_0 + dt F'(u_n) (Phi_1 + Phi_2)
    dL/du_{n-1} += -dt F'(u_{n-1}) Phi_2
    dL/dalpha   += dt <Phi_1 + Phi_2, u_n (1 - u_n/K)> - dt <Phi_2, u_{n-1} (1 - u_{n-1}/K)>
beta: by Eq. 3.10 the step is y(1) of y' = A y + v_1 + t v_2, y(0) = u_n, so
    dL = int_0^1 mu(t)^T dA y(t) dt,  mu(t) = e^{(1-t) A} lambda,
    y(t) = phi_0(tA) u_n + phi_1(tA) (t v_1) + phi_2(tA) (t^2 v_2),
evaluated with Gauss-Legendre in t.  With (C u)_p = h^-2 [sum_{q comp} beta_pq
(u_q - u_p) - sum_ghost beta_f (1 - w_f) u_p]:
    d(mu^T C y)/d beta_pq = -h^-2 (mu_p - mu_q)(y_p - y_q)   (both points computational)
    d(mu^T C y)/d beta_f  = -h^-2 (1 - w_f) mu_p y_p          (face to a ghost point)
and beta_f = (beta_p + beta_q)/2 passes half of each face derivative to each
end node (ghost nodes included).
Parity: pinned by central finite differences of the full trajectory loss
(tests/test_oracle_adjoint.py).
"""
import numpy as np

from . import krylov, phi
from .eb import strides


def reaction_ak(u, alpha, K):
    return alpha * u * (1.0 - u / K)


def reaction_ak_du(u, alpha, K):
    return alpha * (1.0 - 2.0 * u / K)


def reaction_ak_dalpha(u, K):
    return u * (1.0 - u / K)


def gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


class PhiEval:
    """phi-combinations of A = s C for a fixed operator: exact (dense expm) for
    small grids or the adaptive Krylov oracle."""

    def __init__(self, op, exact, tol=1e-12, m_max=40):
        self.op = op
        self.exact = exact
        self.tol = tol
        self.m_max = m_max
        self.Cd = op.C.toarray() if exact else None

    def comb(self, s, vs):
        if self.exact:
            return phi.combination_expm(s * self.Cd, vs)
        C = self.op.C
        y, _ = krylov.phipm(lambda x: s * (C @ x), vs, self.tol, self.m_max, s * self.op.gershgorin())
        return y


def forward(op, u0, dt, nsteps, alpha, K, pe):
    """ETD2 trajectory on computational points; returns the list u_0..u_N."""
    us = [np.array(u0, dtype=np.float64)]
    F_prev = reaction_ak(us[0], alpha, K)
    for _ in range(nsteps):
        u = us[-1]
        F = reaction_ak(u, alpha, K)
        us.append(pe.comb(dt, [u, dt * F, dt * (F - F_prev)]))
        F_prev = F
    return us


def beta_contract(op, mu, y):
    """Node-field gradient of mu^T C(beta) y with beta_f = (beta_p + beta_q)/2."""
    grid = op.grid
    st = strides(grid.n)
    g = np.zeros(grid.size)
    h2 = grid.h * grid.h
    p = op.index
    mu_g = op.to_grid(mu).ravel()
    y_g = op.to_grid(y).ravel()
    comp = op.comp.ravel()
    for d in range(grid.ndim):
        for si, s in enumerate((-1, 1)):
            face = 2 * d + si
            q = p + s * st[d]
            qc = comp[q]
            df = np.where(qc, -(mu_g[p] - mu_g[q]) * (y_g[p] - y_g[q]),
                          -(1.0 - op.weights[:, face]) * mu_g[p] * y_g[p]) / h2
            # a face between two computational points is visited from both
            # ends: each end takes its half once; a ghost face is visited once
            np.add.at(g, p, 0.5 * df)
            gh = ~qc
            np.add.at(g, q[gh], 0.5 * df[gh])
    return g.reshape(grid.n)


def adjoint_step(op, pe, dt, u_n, u_nm1, lam, alpha, K, nquad):
    """Contributions of one ETD2 step.  Returns (to_u_n, to_u_nm1, dalpha,
    dbeta_grid)."""
    P0 = pe.comb(dt, [lam, 0 * lam, 0 * lam])
    P1 = pe.comb(dt, [0 * lam, lam, 0 * lam])
    P2 = pe.comb(dt, [0 * lam, 0 * lam, lam])
    to_n = P0 + dt * reaction_ak_du(u_n, alpha, K) * (P1 + P2)
    to_nm1 = -dt * reaction_ak_du(u_nm1, alpha, K) * P2
    dalpha = dt * np.dot(P1 + P2, reaction_ak_dalpha(u_n, K)) - dt * np.dot(P2, reaction_ak_dalpha(u_nm1, K))
    F = reaction_ak(u_n, alpha, K)
    Fm = reaction_ak(u_nm1, alpha, K)
    v1, v2 = dt * F, dt * (F - Fm)
    ts, ws = gauss_legendre01(nquad)
    gb = np.zeros(op.grid.n)
    for t, w in zip(ts, ws):
        y = pe.comb(t * dt, [u_n, t * v1, t * t * v2])
        mu = pe.comb((1.0 - t) * dt, [lam, 0 * lam, 0 * lam])
        gb += (w * dt) * beta_contract(op, mu, y)
    return to_n, to_nm1, dalpha, gb


def trajectory_gradient(op, u0, dt, nsteps, alpha, K, target, pe, nquad):
    """Loss L = 1/2 |u_N - target|^2 (computational points) and its gradients
    with respect to u_0 (computational points), beta (grid) and alpha."""
    us = forward(op, u0, dt, nsteps, alpha, K, pe)
    r = us[-1] - target
    L = 0.5 * float(np.dot(r, r))
    lam = r.copy()
    acc = np.zeros_like(lam)
    gbeta = np.zeros(op.grid.n)
    galpha = 0.0
    for n in range(nsteps - 1, -1, -1):
        u_n = us[n]
        u_nm1 = us[n - 1] if n > 0 else us[0]
        to_n, to_nm1, da, gb = adjoint_step(op, pe, dt, u_n, u_nm1, lam, alpha, K, nquad)
        galpha += da
        gbeta += gb
        lam = to_n + acc
        acc = to_nm1
        if n == 0:
            lam = lam + acc  # u_{-1} is u_0
    return L, lam, gbeta, galpha
