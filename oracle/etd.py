"""Reaction terms and the ETD1 / ETD2 / ETD2RK / ETD3RK / ETD4RK steps (Sec. 3,
Eq. 3.1-3.3, the ETD1 / ETD2 formulas of Sec. 3.1 and the Runge-Kutta forms
of Sec. 3.2), on a fixed embedded-boundary domain.

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
ETD3RK and ETD4RK (Sec. 3.2): the paper's stages in its order, each written as
one combination using U + h phi_1(h C) C U = phi_0(h C) U.  The paper's phi_k
are those of Eq. 3.7, phi_k(z) = int_0^1 e^{(1-l) z} l^{k-1} dl, so its phi_3
is twice the standard phi_3 (which carries 1 / 2!); the paper's recursion,
Eq. 3.8, confirms that normalisation.  The combinations here use the standard
phi_k, so the phi_3 vector of the final stage is the paper's times two.
Multistep ETD3 (Eq. 3.8b with s = 3): the weights g_m are defined by integrals,
so they do not depend on the phi normalisation; with the standard phi_k,
g_0 = phi_1, g_1 = phi_2 and g_2 = phi_3 + phi_2 / 2 (the binomial
(-lambda choose 2) = lambda (lambda + 1) / 2).  With the backward differences
of F this is one combination:
    v_0 = U_n, v_1 = dt F_n, v_2 = dt (3/2 F_n - 2 F_{n-1} + 1/2 F_{n-2}),
    v_3 = dt (F_n - 2 F_{n-1} + F_{n-2}).
Start-up (a reading, extending the ETD2 one): with one earlier F the step is
ETD2, with none it is ETD1.
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
    """sum_k phi_k(dt C) v_k, k = 0 .. len(vs) - 1, standard phi_k (Eq. 3.9):
    the dense augmented expm (exact=True, small grids) or the adaptive Krylov
    phipm.  Returns (y, trace)."""
    if exact:
        return phi.combination_expm(dt * op.C.toarray(), vs), []
    C = op.C
    return krylov.phipm(lambda x: dt * (C @ x), vs, tol, m_max, dt * op.gershgorin(), forced_trace=forced_trace)


def etd1_step(op, u_n, F_n, dt, tol=1e-10, m_max=40, exact=False, forced_trace=None):
    """One ETD1 step: U_{n+1} = phi_0(dt C) U_n + dt phi_1(dt C) F_n."""
    return combination(op, [u_n, dt * F_n, np.zeros_like(u_n)], dt, tol, m_max, exact, forced_trace)


def _ft(forced, i):
    """Decision trace of the i-th combination of a step (None: decide)."""
    return None if forced is None else forced[i]


def etd2rk_step(op, u_n, F_of, t_n, dt, tol=1e-10, m_max=40, exact=False, forced_traces=None):
    """One ETD2RK step (Sec. 3.2).  F_of(U, t) -> F vector.  Returns
    (U_{n+1}, a_n, (trace of the first combination, trace of the second)).
    forced_traces: None, or one decision trace per combination to replay."""
    F_n = F_of(u_n, t_n)
    a, tr1 = etd1_step(op, u_n, F_n, dt, tol, m_max, exact, _ft(forced_traces, 0))
    z = np.zeros_like(u_n)
    d, tr2 = combination(op, [z, z, dt * (F_of(a, t_n + dt) - F_n)], dt, tol, m_max, exact, _ft(forced_traces, 1))
    return a + d, a, (tr1, tr2)


def etd3rk_step(op, u_n, F_of, t_n, dt, tol=1e-10, m_max=40, exact=False, forced_traces=None):
    """One ETD3RK step (Sec. 3.2).  Returns (U_{n+1}, (a_n, b_n), traces).
    forced_traces: None, or one decision trace per combination to replay."""
    z = np.zeros_like(u_n)
    F_n = F_of(u_n, t_n)
    # a_n = U_n + dt/2 phi_1(dt C / 2)(F_n + C U_n)
    a, tr_a = combination(op, [u_n, 0.5 * dt * F_n, z], 0.5 * dt, tol, m_max, exact, _ft(forced_traces, 0))
    F_a = F_of(a, t_n + 0.5 * dt)
    # b_n = U_n + dt phi_1(dt C)(C U_n + 2 F(a_n) - F_n)
    b, tr_b = combination(op, [u_n, dt * (2.0 * F_a - F_n), z], dt, tol, m_max, exact, _ft(forced_traces, 1))
    F_b = F_of(b, t_n + dt)
    # U_{n+1} = U_n + dt phi_1 (C U_n + F_n) + dt phi_2 (-3 F_n + 4 F(a_n) - F(b_n))
    #         + dt phi_3 (2 F_n - 4 F(a_n) + 2 F(b_n)),  the paper's phi_3 = 2 x standard
    v2 = dt * (-3.0 * F_n + 4.0 * F_a - F_b)
    v3 = 2.0 * dt * (2.0 * F_n - 4.0 * F_a + 2.0 * F_b)
    u, tr_u = combination(op, [u_n, dt * F_n, v2, v3], dt, tol, m_max, exact, _ft(forced_traces, 2))
    return u, (a, b), (tr_a, tr_b, tr_u)


def etd4rk_step(op, u_n, F_of, t_n, dt, tol=1e-10, m_max=40, exact=False, forced_traces=None):
    """One ETD4RK step (Sec. 3.2).  Returns (U_{n+1}, (a_n, b_n, c_n), traces).
    forced_traces: None, or one decision trace per combination to replay."""
    z = np.zeros_like(u_n)
    h2 = 0.5 * dt
    F_n = F_of(u_n, t_n)
    # a_n = U_n + dt/2 phi_1(dt C / 2)(F_n + C U_n)
    a, tr_a = combination(op, [u_n, h2 * F_n, z], h2, tol, m_max, exact, _ft(forced_traces, 0))
    F_a = F_of(a, t_n + h2)
    # b_n = U_n + dt/2 phi_1(dt C / 2)(F(a_n) + C U_n)
    b, tr_b = combination(op, [u_n, h2 * F_a, z], h2, tol, m_max, exact, _ft(forced_traces, 1))
    F_b = F_of(b, t_n + h2)
    # c_n = a_n + dt/2 phi_1(dt C / 2)(2 F(b_n) - F_n + C a_n)
    c, tr_c = combination(op, [a, h2 * (2.0 * F_b - F_n), z], h2, tol, m_max, exact, _ft(forced_traces, 2))
    F_c = F_of(c, t_n + dt)
    # U_{n+1} = U_n + dt phi_1 (C U_n + F_n)
    #         + dt phi_2 (-3 F_n + 2 (F(a_n) + F(b_n)) - F(c_n))
    #         + dt phi_3 (2 F_n - 2 (F(a_n) + F(b_n)) + 2 F(c_n)),  the paper's phi_3 = 2 x standard
    v2 = dt * (-3.0 * F_n + 2.0 * (F_a + F_b) - F_c)
    v3 = 2.0 * dt * (2.0 * F_n - 2.0 * (F_a + F_b) + 2.0 * F_c)
    u, tr_u = combination(op, [u_n, dt * F_n, v2, v3], dt, tol, m_max, exact, _ft(forced_traces, 3))
    return u, (a, b, c), (tr_a, tr_b, tr_c, tr_u)


def etd3_vectors(u_n, F_n, F_nm1, F_nm2, dt):
    """(v_0, v_1, v_2, v_3) of the multistep ETD3 step (Eq. 3.8b, s = 3)."""
    return [u_n, dt * F_n, dt * (1.5 * F_n - 2.0 * F_nm1 + 0.5 * F_nm2), dt * (F_n - 2.0 * F_nm1 + F_nm2)]


def etd3_step(op, u_n, F_n, F_nm1, F_nm2, dt, tol=1e-10, m_max=40, exact=False, forced_trace=None):
    """One multistep ETD3 step.  Returns (U_{n+1}, trace)."""
    return combination(op, etd3_vectors(u_n, F_n, F_nm1, F_nm2, dt), dt, tol, m_max, exact, forced_trace)


def run_fixed_domain(op, u0, dt, nsteps, F_of, tol=1e-10, m_max=40, exact=False, scheme="etd2"):
    """nsteps steps of `scheme` (etd1, etd2, etd2rk, etd3rk, etd4rk or etd3) on a fixed domain.
    F_of(U, t) -> F vector.  Returns U at t = nsteps dt."""
    u = np.array(u0, dtype=np.float64, copy=True)
    F_prev = None
    hist = []  # etd3: F_n, F_{n-1}, F_{n-2}
    t = 0.0
    for _ in range(nsteps):
        if scheme == "etd2rk":
            u, _, _ = etd2rk_step(op, u, F_of, t, dt, tol=tol, m_max=m_max, exact=exact)
        elif scheme in ("etd3rk", "etd4rk"):
            step = etd3rk_step if scheme == "etd3rk" else etd4rk_step
            u, _, _ = step(op, u, F_of, t, dt, tol=tol, m_max=m_max, exact=exact)
        elif scheme == "etd3":
            F_n = F_of(u, t)
            hist.insert(0, F_n)
            if len(hist) >= 3:
                u, _ = etd3_step(op, u, hist[0], hist[1], hist[2], dt, tol=tol, m_max=m_max, exact=exact)
            else:
                u, _ = etd2_step(op, u, hist[0], hist[-1], dt, tol=tol, m_max=m_max, exact=exact)
            del hist[3:]
        else:
            F_n = F_of(u, t)
            if F_prev is None or scheme == "etd1":
                F_prev = F_n
            u, _ = etd2_step(op, u, F_n, F_prev, dt, tol=tol, m_max=m_max, exact=exact)
            F_prev = F_n
        t += dt
    return u
