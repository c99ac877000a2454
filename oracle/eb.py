"""Embedded-boundary discretisation of div(beta grad u) with interior ghost
points (Sec. 2, Eq. central_difference, Eq. DirichletLineByLine,
Eq. central_difference2, Eq. rbf_ubp).

Point classes (Sec. 2, definitions of interior ghost / computational points):
  inside         phi < 0 (phi == 0 counts as outside -- a reading, the paper
                 only says phi < 0 inside and phi > 0 outside, Sec. 4.3)
  ghost          inside, and at least one of the 2N axis neighbours outside
  computational  inside, and all 2N axis neighbours inside
Unknowns live at computational points only.

Row of computational point p, face (d, s) to neighbour q = p + s e_d, face
coefficient beta_f:
  Case 1  q computational: beta_f (u_q - u_p) / h^2   (Eq. central_difference)
  Case 2  q ghost and r = q + s e_d outside: the interface crosses the grid
          line between q and r.  Lagrange interpolation through (p, u_p) and
          (Gamma, u_Gamma) gives u_q = g_1 u_p + g_G u_Gamma with
          theta = phi_q / (phi_q - phi_r) (one secant step on node values),
          g_1 = theta/(1+theta), g_G = 1/(1+theta)  (Eq. DirichletLineByLine)
  Case 3  q ghost and r inside: u_q from an RBF + linear-tail interpolant
          through x_p and the closest boundary points Gamma1 (of q) and
          Gamma2 (of p) (Eq. rbf_ubp).  With three non-collinear centres the
          tail conditions force lambda = 0, so the rule is the affine
          (barycentric) interpolant; the oracle nevertheless solves the 6x6
          saddle system with a multiquadric psi.  For N >= 3 the paper's
          3-centre system is singular; the reading used is the affine
          function that vanishes on the hyperplane through Gamma1, Gamma2
          with normal n = normalise(nbar - (nbar.t) t),
          nbar = normalise(grad phi(x_q) + grad phi(x_p)),
          t = (Gamma2 - Gamma1)/|Gamma2 - Gamma1|, giving
          w = ((x_q - Gamma1).n) / ((x_p - Gamma1).n).
In both ghost cases u_q = w u_p + (boundary data), so the face contributes
-beta_f (1 - w) u_p to the diagonal and beta_f (data) / h^2 to the right-hand
side; off-diagonals are untouched and C stays symmetric (Sec. 2, remarks
after Eq. central_difference2 and Eq. rbf_ubp).  w is clamped to [0, 1].

Face coefficient: a scalar beta; a node field beta -> (beta_p + beta_q)/2;
an analytic beta(x) -> beta at the face midpoint.
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid

DOMAIN_MARGIN = 3  # inside nodes must keep this many nodes from the box edge


class DomainError(ValueError):
    pass


def strides(n):
    s = [1] * len(n)
    for d in range(len(n) - 2, -1, -1):
        s[d] = s[d + 1] * n[d + 1]
    return s


def classify(grid: Grid, phi):
    """Inside / ghost / computational masks (Sec. 2)."""
    phi = np.asarray(phi, dtype=np.float64)
    inside = phi < 0.0
    all_nb_inside = inside.copy()
    for d in range(grid.ndim):
        for s in (-1, 1):
            nb = np.zeros_like(inside)
            src = [slice(None)] * grid.ndim
            dst = [slice(None)] * grid.ndim
            if s > 0:
                src[d], dst[d] = slice(1, None), slice(0, -1)
            else:
                src[d], dst[d] = slice(0, -1), slice(1, None)
            nb[tuple(dst)] = inside[tuple(src)]
            all_nb_inside &= nb
    comp = inside & all_nb_inside
    ghost = inside & ~comp
    edge = np.zeros_like(inside)
    for d in range(grid.ndim):
        sl = [slice(None)] * grid.ndim
        sl[d] = slice(0, DOMAIN_MARGIN)
        edge[tuple(sl)] = True
        sl[d] = slice(grid.n[d] - DOMAIN_MARGIN, None)
        edge[tuple(sl)] = True
    if np.any(inside & edge):
        raise DomainError("inside node within %d nodes of the box edge" % DOMAIN_MARGIN)
    return inside, ghost, comp


def _node_coords(grid, flat):
    idx = np.unravel_index(flat, grid.n)
    return np.stack([grid.lo[d] + grid.h * idx[d] for d in range(grid.ndim)], axis=-1)


def _grad_phi_nodes(grid, phi, flat):
    """Central-difference gradient of the node values of phi at flat indices."""
    st = strides(grid.n)
    pf = phi.ravel()
    g = np.empty((len(flat), grid.ndim))
    for d in range(grid.ndim):
        g[:, d] = (pf[flat + st[d]] - pf[flat - st[d]]) / (2.0 * grid.h)
    return g


def _closest_points(x, phi_x, grad_x, phi_fn=None):
    """Closest boundary point x - phi grad / |grad|^2 (one projection step on
    node data), or the projection iterated to convergence with the analytic
    level set phi_fn(x) -> (phi, grad) when one is given."""
    if phi_fn is None:
        g2 = np.sum(grad_x * grad_x, axis=-1)
        return x - (phi_x / g2)[:, None] * grad_x
    y = x.copy()
    for _ in range(50):
        f, g = phi_fn(y)
        g2 = np.sum(g * g, axis=-1)
        y = y - (f / g2)[:, None] * g
        if np.max(np.abs(f)) < 1e-15:
            break
    return y


def multiquadric(r, h):
    return np.sqrt(r * r + h * h)


def rbf_weights_2d(xp, xq, g1, g2, h):
    """Coefficients (c_p, c_G1, c_G2) with u_q = c_p u_p + c_G1 u_G1 + c_G2 u_G2,
    from the RBF + linear-tail interpolant of Eq. rbf_ubp: solve the 6x6
    saddle system B and evaluate (psi_q, p_q)^T B^{-1} (u, 0)."""
    centres = np.stack([xp, g1, g2])
    dist = np.sqrt(np.sum((centres[:, None, :] - centres[None, :, :]) ** 2, axis=-1))
    A = multiquadric(dist, h)
    Pi = np.vstack([np.ones(3), centres[:, 0], centres[:, 1]])
    B = np.zeros((6, 6))
    B[:3, :3] = A
    B[:3, 3:] = Pi.T
    B[3:, :3] = Pi
    psi_q = multiquadric(np.sqrt(np.sum((centres - xq) ** 2, axis=-1)), h)
    poly_q = np.array([1.0, xq[0], xq[1]])
    c = np.linalg.solve(B.T, np.concatenate([psi_q, poly_q]))
    return c[:3]


class EBOperator:
    """The discrete operator C on computational points (U_t = C U + ..., Eq. 3.2).

    Attributes
      comp, ghost, inside : boolean masks on the grid
      index   : flat grid indices of the computational points in C order
      C       : scipy.sparse CSR matrix, C[i, j] for computational points i, j
      diag    : D_p with C_pp = -D_p / h^2
      brow, bcoef, bpts, bcase : boundary-data terms, b_i = sum bcoef * u_Gamma(bpts)
      nclamp  : number of ghost weights clamped to [0, 1]
      kinds   : per (row, face) case, for tests: array of shape (ncomp, 2N)
      weights : per (row, face) ghost weight w (1 for case 1 faces)
    """

    def __init__(self, grid, phi, beta, phi_fn=None, boundary_data=False):
        self.grid = grid
        phi = np.asarray(phi, dtype=np.float64)
        self.phi = phi
        self.inside, self.ghost, self.comp = classify(grid, phi)
        self.index = np.flatnonzero(self.comp.ravel())
        self.ncomp = len(self.index)
        N, h = grid.ndim, grid.h
        st = strides(grid.n)
        ordinal = -np.ones(grid.size, dtype=np.int64)
        ordinal[self.index] = np.arange(self.ncomp)
        pf = phi.ravel()
        inside_f = self.inside.ravel()
        comp_f = self.comp.ravel()
        p = self.index
        xp = _node_coords(grid, p)
        rows, cols, vals = [], [], []
        diag = np.zeros(self.ncomp)
        self.kinds = np.zeros((self.ncomp, 2 * N), dtype=np.int8)
        self.weights = np.ones((self.ncomp, 2 * N))
        brow, bcoef, bpts, bcase = [], [], [], []
        nclamp = 0
        for d in range(N):
            for si, s in enumerate((-1, 1)):
                face = 2 * d + si
                q = p + s * st[d]
                bf = self._face_beta(beta, p, q, xp, d, s)
                diag += bf
                qc = comp_f[q]
                # Case 1: neighbour is a computational point.
                rows.append(np.arange(self.ncomp)[qc])
                cols.append(ordinal[q[qc]])
                vals.append(bf[qc] / (h * h))
                self.kinds[qc, face] = 1
                # Ghost faces.
                gi = np.flatnonzero(~qc)
                if len(gi) == 0:
                    continue
                assert np.all(inside_f[q[gi]]), "a computational point has an outside neighbour"
                r = q[gi] + s * st[d]
                case2 = pf[r] >= 0.0
                w = np.empty(len(gi))
                # Case 2: line-by-line Lagrange interpolation.
                i2 = gi[case2]
                phq, phr = pf[q[i2]], pf[r[case2]]
                theta = phq / (phq - phr)
                w[case2] = theta / (1.0 + theta)
                self.kinds[i2, face] = 2
                if boundary_data:
                    xq = _node_coords(grid, q[i2])
                    xg = xq.copy()
                    xg[:, d] += s * theta * h
                    brow.append(i2)
                    bcoef.append(bf[i2] * (1.0 / (1.0 + theta)) / (h * h))
                    bpts.append(xg)
                    bcase.append(np.full(len(i2), 2))
                # Case 3: RBF (N = 2) / hyperplane (N >= 3) interpolation.
                i3 = gi[~case2]
                if len(i3):
                    w3, bdat = self._case3(grid, phi, p[i3], q[i3], phi_fn, boundary_data)
                    w[~case2] = w3
                    self.kinds[i3, face] = 3
                    if boundary_data:
                        for (cb, pts) in bdat:
                            brow.append(i3)
                            bcoef.append(bf[i3] * cb / (h * h))
                            bpts.append(pts)
                            bcase.append(np.full(len(i3), 3))
                wc = np.clip(w, 0.0, 1.0)
                nclamp += int(np.count_nonzero(wc != w))
                self.weights[gi, face] = wc
                diag[gi] -= bf[gi] * wc
        self.diag = diag
        self.nclamp = nclamp
        rows.append(np.arange(self.ncomp))
        cols.append(np.arange(self.ncomp))
        vals.append(-diag / (h * h))
        self.C = sp.csr_matrix(
            (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
            shape=(self.ncomp, self.ncomp),
        )
        if boundary_data and brow:
            self.brow = np.concatenate(brow)
            self.bcoef = np.concatenate(bcoef)
            self.bpts = np.concatenate(bpts)
            self.bcase = np.concatenate(bcase)
        else:
            self.brow = np.zeros(0, dtype=np.int64)
            self.bcoef = np.zeros(0)
            self.bpts = np.zeros((0, N))
            self.bcase = np.zeros(0, dtype=np.int64)

    # face coefficient between p and q = p + s e_d
    def _face_beta(self, beta, p, q, xp, d, s):
        grid = self.grid
        if callable(beta):
            mid = xp.copy()
            mid[:, d] += 0.5 * s * grid.h
            return np.asarray(beta(mid), dtype=np.float64)
        b = np.asarray(beta, dtype=np.float64)
        if b.ndim == 0:
            return np.full(len(p), float(b))
        bf = b.ravel()
        return 0.5 * (bf[p] + bf[q])

    def _case3(self, grid, phi, p, q, phi_fn, boundary_data):
        N, h = grid.ndim, grid.h
        xp = _node_coords(grid, p)
        xq = _node_coords(grid, q)
        if phi_fn is None:
            pf = phi.ravel()
            php, phq = pf[p], pf[q]
            gp = _grad_phi_nodes(grid, phi, p)
            gq = _grad_phi_nodes(grid, phi, q)
        else:
            php, gp = phi_fn(xp)
            phq, gq = phi_fn(xq)
        G1 = _closest_points(xq, phq, gq, phi_fn)   # closest to the ghost point
        G2 = _closest_points(xp, php, gp, phi_fn)   # closest to the computational point
        w = np.empty(len(p))
        cG1 = np.zeros(len(p))
        cG2 = np.zeros(len(p))
        if N == 2:
            for k in range(len(p)):
                e1 = G1[k] - xp[k]
                e2 = G2[k] - xp[k]
                det = e1[0] * e2[1] - e1[1] * e2[0]
                if abs(det) < 1e-12 * h * h:
                    w[k] = phq[k] / php[k]
                    cG1[k] = 1.0 - w[k]
                    continue
                c = rbf_weights_2d(xp[k], xq[k], G1[k], G2[k], h)
                w[k], cG1[k], cG2[k] = c
        else:
            nb = gq + gp
            nb = nb / np.linalg.norm(nb, axis=-1, keepdims=True)
            t = G2 - G1
            tl = np.linalg.norm(t, axis=-1)
            n = nb.copy()
            ok = tl >= 1e-12 * h
            tt = t[ok] / tl[ok][:, None]
            n[ok] = nb[ok] - np.sum(nb[ok] * tt, axis=-1)[:, None] * tt
            n[ok] = n[ok] / np.linalg.norm(n[ok], axis=-1, keepdims=True)
            num = np.sum((xq - G1) * n, axis=-1)
            den = np.sum((xp - G1) * n, axis=-1)
            degen = np.abs(den) < 1e-12 * h
            w = np.where(degen, phq / np.where(degen, php, 1.0), num / np.where(degen, 1.0, den))
            cG1 = 1.0 - w
            if boundary_data:
                raise NotImplementedError("nonzero boundary data in case 3 is defined for N = 2 only")
        return w, [(cG1, G1), (cG2, G2)]

    # ---- helpers -------------------------------------------------------
    def boundary_rhs(self, u_gamma):
        """b_i = sum over boundary terms of row i of bcoef * u_gamma(point)."""
        b = np.zeros(self.ncomp)
        if len(self.brow):
            np.add.at(b, self.brow, self.bcoef * u_gamma(self.bpts))
        return b

    def to_grid(self, v, fill=0.0):
        out = np.full(self.grid.size, fill)
        out[self.index] = v
        return out.reshape(self.grid.n)

    def from_grid(self, a):
        return np.asarray(a, dtype=np.float64).ravel()[self.index]

    def gershgorin(self):
        """max_i sum_j |C_ij| (an upper bound on the spectral radius of C)."""
        return float(np.max(np.asarray(abs(self.C).sum(axis=1)).ravel()))
