"""Adaptive Krylov evaluation of y = sum_{k=0}^p phi_k(A) v_k (Sec. 3.3, Eq. 3.9),
time-stepping the equivalent ODE of Eq. 3.10,

    y'(t) = A y + sum_{k=1}^p t^{k-1}/(k-1)! v_k,   y(0) = v_0,   y = y(1).

The paper names phipm_simul_iom2 (Luan, Pudykiewicz & Reynolds 2019) and does
not print it; this is a restatement of that family (Niesen & Wright's phipm
with incomplete orthogonalisation against the two previous basis vectors).
Readings for what the paper leaves open (controller constants are this
implementation's, and are shared with the CUDA path through this
specification only, not through code):

Substep from t_k with step tau (phipm):
  w_0 = y(t_k),  w_j = A w_{j-1} + sum_{l=0}^{p-j} t_k^l / l! v_{j+l}
  y(t_k + tau) = sum_{j=0}^{p-1} tau^j / j! w_j + tau^p phi_p(tau A) w_p
phi_p(tau A) w_p ~ beta V_m phi_p(tau H_m) e_1 with beta = |w_p|, from an
IOM2 (Lanczos) basis: z = A v_j, h_jj = <z, v_j>, h_{j-1,j} = <z, v_{j-1}>,
z -= h_jj v_j + h_{j-1,j} v_{j-1}, h_{j+1,j} = |z|, v_{j+1} = z / h_{j+1,j}.
The small functions come from the exponential of the augmented matrix
[[tau H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]] (size m+p+1); the a-posteriori
error estimate is err = tau^{p+1} beta h_{m+1,m} |e_m^T phi_{p+1}(tau H_m) e_1|.
Control: tau = 1 at the start of a call; the basis grows to m_max with a check
every 5 vectors and at m_max; a check accepts when err <= tol tau |y(t_k)|_2
(|y| is replaced by max(|y(t_k)|, |v_1|, ..., |v_p|, 1e-300) so that a
combination with v_0 = 0, a single phi_k acting on a vector, still has a
nonzero scale).  Happy breakdown (h_{j+1,j} < 1e-12 anorm)
accepts at once.  A failed check at m_max shrinks
tau <- tau max(0.2, 0.9 (tol tau |y| / err)^{1/(m+1)}) reusing the basis,
until accepted or tau < 1e-6 (error).  After acceptance
tau_next = min(1 - t, tau min(2, 0.9 (tol tau |y| / err)^{1/(m+1)})).
If tau was the whole remaining interval the substep ends exactly at t = 1.
w_p = 0 accepts tau = 1 - t_k with no basis.
"""
import math

import numpy as np

from .phi import phi_columns_expm

CHECK_EVERY = 5
TAU_MIN = 1e-6
BREAKDOWN_REL = 1e-12


class KrylovError(RuntimeError):
    pass


def phipm(apply_A, vs, tol, m_max, anorm, forced_trace=None, dot=None):
    """Returns (y, trace); trace lists (tau, m, rejections) per accepted substep.

    forced_trace, if given, replays a decision trace instead of deciding:
    substep k uses step forced_trace[k][0] and basis size forced_trace[k][1]
    (to compare two implementations whose error estimates straddle a
    threshold; the arithmetic is unchanged)."""
    if dot is None:
        dot = np.dot
    p = len(vs) - 1
    assert p >= 1
    y = np.array(vs[0], dtype=np.float64, copy=True)
    vscale = max(math.sqrt(dot(v, v)) for v in vs[1:])
    t = 0.0
    tau = 1.0
    trace = []
    k = 0
    while t < 1.0:
        last = tau >= 1.0 - t
        if last:
            tau = 1.0 - t
        if forced_trace is not None:
            tau = forced_trace[k][0]
            last = k == len(forced_trace) - 1
        # w_0 .. w_p
        w = [y]
        for j in range(1, p + 1):
            wj = apply_A(w[j - 1])
            for l in range(0, p - j + 1):
                wj = wj + (t ** l / math.factorial(l)) * vs[j + l]
            w.append(wj)
        ynorm = max(math.sqrt(dot(y, y)), vscale, 1e-300)
        beta = math.sqrt(dot(w[p], w[p]))
        if beta == 0.0:
            y = sum((tau ** j / math.factorial(j)) * w[j] for j in range(p))
            trace.append((tau, 0, 0))
            t = 1.0 if last else t + tau
            tau = min(1.0 - t, 2.0 * tau) if t < 1.0 else tau
            k += 1
            continue
        # IOM2 / Lanczos basis, classical Gram-Schmidt against v_j, v_{j-1}
        V = [w[p] / beta]
        H = np.zeros((m_max + 1, m_max))
        m_forced = forced_trace[k][1] if forced_trace is not None else None
        accepted = False
        err = None
        m = 0
        for j in range(m_max):
            z = apply_A(V[j])
            H[j, j] = dot(z, V[j])
            if j > 0:
                H[j - 1, j] = dot(z, V[j - 1])
                z = z - H[j, j] * V[j] - H[j - 1, j] * V[j - 1]
            else:
                z = z - H[j, j] * V[j]
            H[j + 1, j] = math.sqrt(dot(z, z))
            m = j + 1
            breakdown = H[j + 1, j] < BREAKDOWN_REL * anorm
            if not breakdown:
                V.append(z / H[j + 1, j])
            if m_forced is not None:
                if m == m_forced or breakdown:
                    err = 0.0 if breakdown else _estimate(H, m, tau, beta, p)
                    accepted = True
                    break
                continue
            if m % CHECK_EVERY == 0 or m == m_max or breakdown:
                err = 0.0 if breakdown else _estimate(H, m, tau, beta, p)
                if err <= tol * tau * ynorm:
                    accepted = True
                    break
        rejections = 0
        if not accepted:
            while err > tol * tau * ynorm:
                fac = max(0.2, 0.9 * (tol * tau * ynorm / err) ** (1.0 / (m + 1)))
                tau = tau * fac
                last = False
                rejections += 1
                if tau < TAU_MIN:
                    raise KrylovError("tolerance not met at tau_min")
                err = _estimate(H, m, tau, beta, p)
        # combination
        cols = phi_columns_expm(tau * H[:m, :m], p + 1)
        coef = beta * cols[:, p - 1]
        ynew = sum((tau ** j / math.factorial(j)) * w[j] for j in range(p))
        ynew = ynew + (tau ** p) * sum(coef[i] * V[i] for i in range(m))
        trace.append((tau, m, rejections))
        if err == 0.0:
            grow = 2.0
        else:
            grow = min(2.0, 0.9 * (tol * tau * ynorm / err) ** (1.0 / (m + 1)))
        y = ynew
        t = 1.0 if last else t + tau
        tau = min(1.0 - t, tau * grow) if t < 1.0 else tau
        k += 1
    return y, trace


def _estimate(H, m, tau, beta, p):
    cols = phi_columns_expm(tau * H[:m, :m], p + 1)
    return (tau ** (p + 1)) * beta * H[m, m - 1] * abs(cols[m - 1, p])
