"""phi-functions and the exact linear combination sum_k phi_k(A) v_k
(Sec. 3.1 Eq. 3.7 / Eq. 3.8, Sec. 3.3 Eq. 3.9 and the equivalent ODE Eq. 3.10).

Normalisation.  Eq. 3.7 writes phi_k(z) = int_0^1 e^{(1-l)z} l^{k-1} dl and the
recursion of Eq. 3.8 is phi_{k+1} = (k phi_k - 1)/z; the ODE of Eq. 3.10 uses
t^{k-1}/(k-1)!.  The two agree for k <= 2, which is all ETD1/ETD2 need.  This
module uses the standard normalisation phi_k(z) = sum_{i>=0} z^i/(i+k)!,
whose recursion is phi_{k+1}(z) = (phi_k(z) - 1/k!)/z, so that Eq. 3.10 holds
for every p (a reading).

Two independent exact evaluations for small matrices:
  combination_expm  -- the augmented matrix [[A, W], [0, J]] with
                       W = [v_p, ..., v_1] and J the p x p upward shift;
                       exp of it applied to [v_0; e_p] gives the sum
                       (the block-triangular identity of Al-Mohy & Higham).
  combination_eig   -- A symmetric: A = Q diag(lam) Q^T, phi_k(A) v =
                       Q phi_k(lam) Q^T v with scalar phi_k.
"""
import math

import numpy as np
import scipy.linalg as sla


def phi_scalar(k, z):
    """phi_k(z) for real z (array), standard normalisation.

    |z| < 1: Taylor series sum_{i>=0} z^i/(i+k)! (40 terms, converges far
    below double rounding); |z| >= 1: phi_0 = e^z and the recursion
    phi_{j+1} = (phi_j - 1/j!)/z."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    acc = np.zeros_like(zs)
    term = np.full_like(zs, 1.0 / math.factorial(k))
    for i in range(40):
        acc = acc + term
        term = term * zs / (i + k + 1)
    out[small] = acc
    zl = z[~small]
    f = np.exp(zl)
    for j in range(k):
        f = (f - 1.0 / math.factorial(j)) / zl
    out[~small] = f
    return out


def augmented(A, vs):
    """[[A, W], [0, J]] with W = [v_p, ..., v_1], J the p x p upward shift."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    p = len(vs) - 1
    M = np.zeros((n + p, n + p))
    M[:n, :n] = A
    for c in range(p):
        M[:n, n + c] = vs[p - c]
    for c in range(p - 1):
        M[n + c, n + c + 1] = 1.0
    return M


def combination_expm(A, vs):
    """sum_{k=0}^p phi_k(A) v_k via the augmented matrix exponential."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    p = len(vs) - 1
    if p == 0:
        return sla.expm(A) @ vs[0]
    M = augmented(A, vs)
    rhs = np.zeros(n + p)
    rhs[:n] = vs[0]
    rhs[n + p - 1] = 1.0
    return (sla.expm(M) @ rhs)[:n]


def combination_eig(A, vs):
    """sum_{k=0}^p phi_k(A) v_k for symmetric A via eigendecomposition."""
    A = np.asarray(A, dtype=np.float64)
    lam, Q = np.linalg.eigh(0.5 * (A + A.T))
    out = np.zeros(A.shape[0])
    for k, v in enumerate(vs):
        out += Q @ (phi_scalar(k, lam) * (Q.T @ v))
    return out


def phi_columns_expm(H, q):
    """[phi_1(H) e1, ..., phi_q(H) e1] from exp([[H, e1 0..0], [0, J_q]])
    (the columns of the top-right block); H is m x m."""
    H = np.asarray(H, dtype=np.float64)
    m = H.shape[0]
    K = np.zeros((m + q, m + q))
    K[:m, :m] = H
    K[0, m] = 1.0
    for i in range(q - 1):
        K[m + i, m + i + 1] = 1.0
    E = sla.expm(K)
    return E[:m, m:m + q]
