"""Embedded-boundary Poisson solve (Sec. 2, the variable-coefficient Poisson
equation div(beta grad u) = f with Dirichlet data, discretised with interior
ghost points; Sec. 4.1 applies it to a virus-shaped domain).

The discrete problem at the computational points is C u + b = f, with C the
matrix of oracle.eb.EBOperator and b the boundary-data term of the ghost
values (EBOperator.boundary_rhs).  The oracle solves it directly (sparse LU):
the plain definition, which the GPU reaches by conjugate gradients on -C
(symmetric positive definite by Sec. 2's construction).  Test infrastructure
only.
"""
import numpy as np
import scipy.sparse.linalg as spla


def solve(op, f, u_gamma=None):
    """u on the computational points from f (per computational point) and the
    boundary data u_gamma (a function of points, or None for zero data)."""
    b = op.boundary_rhs(u_gamma) if u_gamma is not None else np.zeros(op.ncomp)
    return spla.spsolve(op.C.tocsc(), np.asarray(f, dtype=np.float64) - b)
