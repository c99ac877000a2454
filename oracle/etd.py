"""Reaction terms and the ETD1 / ETD2 / ETD2RK steps (Sec. 3, Eq. 3.1-3.3, the
ETD1 / ETD2 formulas of Sec. 3.1 and ETD2RK of Sec. 3.2), on a fixed
embedded-boundary domain.

Semi-discrete system (Eq. 3.2): U_t = C U + F(U, t) with C from oracle.eb.
ETD2 (Cox-Matthews multistep, Sec. 3.1):
    U_{n+1} = phi_0(dt C) U_n + dt phi_1(dt C) F_n + dt phi_2(dt C) (F_n - F_{n-1})
i.e. the combination of Eq. 3.9 with A = dt C, v_0 = U_n, v_1 = dt F_n,
v_2 = dt (F_n - F_{n-1}).  The first step takes F_{-1} = F_0 (a reading), which
makes it exactly ETD1:  U_1 = U_0 + dt phi_1(dt C)(F_0 + C U_0).
ETD2RK (Sec. 3.2):
    a_n     = U_n + dt phi_1(dt C)(F_n + C U_n)      (= the ETD1 step)
    U_{n+1} = U_n + dt phi_1(dt C)(F_n + C U_n) + dt phi_2(dt C)(F(a_n, t_n + dt) - F_n)
            = a_n + dt phi_2(dt C)(F(a_n, t_n + dt) - F_n),
so two combinations: (v_0, v_1, v_2) = (U_n, dt F_n, 0), then (0, 0, dt (F(a_n) - F_n)).
"""
import numpy as np

from . import krylov, phi


def reaction(kind, params, us):
    """F(U) for the reaction families used by the workloads.

    logistic     f(u) = u (1 - u)                                   (Sec. 4.3, a = b = 1)
    logistic_ak  f(u) = alpha u (1 - u / K)    params = (alpha, K)
    competition  f(u, v) = (u (1 - u - a v), r v (1 - v - b u))   params = (a, b, r)
    none         f = 0
    `us` is a list of per-species vectors; returns a list."""
    if kind == "logistic":
        return [u * (1.0 - u) for u in us]
    if kind == "logistic_ak":
        alpha, K = params[0], params[1]
        return [alpha * u * (1.0 - u / K) for u in us]
    if kind == "competition":
        a, b, r = params[0], params[1], params[2]
        u, v = us
        return [u * (1.0 - u - a * v), r * v * (1.0 - v - b * u)]
    if kind == "none":
        return [np.zeros_like(u) for u in us]
    raise ValueError(kind)


def etd2_vectors(u_n, F_n, F_nm1, dt):
    """(v_0, v_1, v_2) of the ETD2 step."""
    return [u_n, dt * F_n, dt * (F_n - F_nm1)]


def etd2_step(op, u_n, F_n, F_nm1, dt, tol=1e-10, m_max=40, exact=False, forced_trace=None):
    """One ETD2 step on the fixed operator `op` (an oracle.eb.EBOperator).
    exact=True evaluates the combination with the dense augmented expm
    (small grids only); otherwise the adaptive Krylov phipm.
    Returns (U_{n+1}, trace)."""
    vs = etd2_vectors(u_n, F_n, F_nm1, dt)
    if exact:
        A = dt * op.C.toarray()
        return phi.combination_expm(A, vs), []
    C = op.C

    def apply_A(x):
        return dt * (C @ x)

    anorm = dt * op.gershgorin()
    return krylov.phipm(apply_A, vs, tol, m_max, anorm, forced_trace=forced_trace)


def combination(op, vs, dt, tol=1e-10, m_max=40, exact=False, forced_trace=None):
    """phi_0(dt C) v_0 + phi_1(dt C) v_1 + phi_2(dt C) v_2 (Eq. 3.9): the dense
    augmented expm (exact=True, small grids) or the adaptive Krylov phipm.
    Returns (y, trace)."""
    if exact:
        return phi.combination_expm(dt * op.C.toarray(), vs), []
    C = op.C
    return krylov.phipm(lambda x: dt * (C @ x), vs, tol, m_max, dt * op.gershgorin(), forced_trace=forced_trace)


def etd1_step(op, u_n, F_n, dt, tol=1e-10, m_max=40, exact=False):
    """One ETD1 step: U_{n+1} = phi_0(dt C) U_n + dt phi_1(dt C) F_n."""
    return combination(op, [u_n, dt * F_n, np.zeros_like(u_n)], dt, tol, m_max, exact)


def etd2rk_step(op, u_n, F_of, t_n, dt, tol=1e-10, m_max=40, exact=False):
    """One ETD2RK step (Sec. 3.2).  F_of(U, t) -> F vector.  Returns
    (U_{n+1}, a_n, (trace of the first combination, trace of the second))."""
    F_n = F_of(u_n, t_n)
    a, tr1 = etd1_step(op, u_n, F_n, dt, tol, m_max, exact)
    z = np.zeros_like(u_n)
    d, tr2 = combination(op, [z, z, dt * (F_of(a, t_n + dt) - F_n)], dt, tol, m_max, exact)
    return a + d, a, (tr1, tr2)


def run_fixed_domain(op, u0, dt, nsteps, F_of, tol=1e-10, m_max=40, exact=False, scheme="etd2"):
    """nsteps steps of `scheme` (etd1, etd2 or etd2rk) on a fixed domain.
    F_of(U, t) -> F vector.  Returns U at t = nsteps dt."""
    u = np.array(u0, dtype=np.float64, copy=True)
    F_prev = None
    t = 0.0
    for _ in range(nsteps):
        if scheme == "etd2rk":
            u, _, _ = etd2rk_step(op, u, F_of, t, dt, tol=tol, m_max=m_max, exact=exact)
        else:
            F_n = F_of(u, t)
            if F_prev is None or scheme == "etd1":
                F_prev = F_n
            u, _ = etd2_step(op, u, F_n, F_prev, dt, tol=tol, m_max=m_max, exact=exact)
            F_prev = F_n
        t += dt
    return u
