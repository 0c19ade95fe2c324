"""Oracle: an independent check of the final result for large n.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The final output of the method is a defined quantity, the N smallest
eigenpairs of A (Algorithm 6 continued to level 0).  For n too large for a
dense eigensolver this module computes the N smallest eigenvalues by a
different algorithm that shares nothing with the hierarchy: shift-invert
Lanczos (ARPACK, scipy.sparse.linalg.eigsh) about sigma = 0 with the exact
inverse from a sparse LU factorisation of A (SuperLU, symmetric ordering on
the pattern of A + A^T, diagonal pivots).  It is the independent check of
the final result where n is above 2000; the tests pin it against dense
LAPACK at small n.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def leftmost_shift_invert(A: sp.spmatrix, N: int, tol: float = 1e-13, ncv: int | None = None):
    """N smallest eigenvalues (ascending) and eigenvectors of the SPD matrix A.

    Eigenvalues of A^{-1} by implicitly restarted Lanczos: lambda = 1 / nu
    for the N largest nu.  ncv defaults to 2 N + 40 Lanczos vectors."""
    A = sp.csc_matrix(A)
    n = A.shape[0]
    lu = sla.splu(A, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True), diag_pivot_thresh=0.0)
    op = sla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.float64)
    k = min(N, n - 1)
    w, V = sla.eigsh(A, k=k, sigma=0.0, which="LM", OPinv=op, tol=tol,
                     ncv=min(n, ncv or (2 * k + 40)))
    o = np.argsort(w, kind="stable")
    return w[o], V[:, o]
