"""Oracle: gradients of eigenpair losses with respect to the CSR values, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no gradient; this is the adjoint of the eigensolver's output.
For a symmetric A with simple eigenpairs (lambda_i, v_i), ||v_i|| = 1:

  d lambda_i = v_i^T dA v_i                           (Hellmann-Feynman)
  d v_i      = -(A - lambda_i I)^+ dA v_i             (first-order perturbation)

so for L(lambda, V) with gl = dL/dlambda and Gv = dL/dV,

  dL/dA = sum_i gl_i v_i v_i^T + sum_i y_i v_i^T,   y_i = -(A - lambda_i I)^+ gv_i.

y_i splits into the part inside the computed block (j <= N, j != i),
  sum_j v_j (v_j^T gv_i) / (lambda_i - lambda_j),
and the part on the complement of the block, z solving
  (A - lambda_i I) z = -(I - V V^T) gv_i   on range(I - V V^T),
which is SPD there when lambda_i < lambda_{N+1}; it is solved by CG on the
projected operator.

Convention: the gradient is reported per stored CSR entry (r, c): G_rc is the
derivative with respect to that entry alone, G_rc = dL/dA[r, c].  A
finite-difference perturbation of a symmetric pair (both entries) therefore
compares with G_rc + G_cr.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads import CSR


def dense_dLdA(A: np.ndarray, N: int, gl: np.ndarray, Gv: np.ndarray | None) -> np.ndarray:
    """Closed form with the full eigen-decomposition (small n only)."""
    lam, V = np.linalg.eigh(A)
    n = A.shape[0]
    G = (V[:, :N] * gl[None, :]) @ V[:, :N].T
    if Gv is not None:
        for i in range(N):
            gi = Gv[:, i]
            if not np.any(gi):
                continue
            y = np.zeros(n)
            for j in range(n):
                if j == i:
                    continue
                y += V[:, j] * (V[:, j] @ gi) / (lam[i] - lam[j])
            G += np.outer(y, V[:, i])
    return G


def projected_cg(A: sp.csr_matrix, V: np.ndarray, sigma: float, rhs: np.ndarray, tol: float = 1e-12,
                 maxit: int = 100000) -> np.ndarray:
    """CG for (A - sigma I) z = rhs on range(I - V V^T) (rhs already in it)."""

    def P(x):
        return x - V @ (V.T @ x)

    def op(x):
        return P(A @ x - sigma * x)

    b = P(rhs)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    bn = np.sqrt(rr)
    if bn == 0:
        return x
    for _ in range(maxit):
        q = op(p)
        a = rr / (p @ q)
        x += a * p
        r -= a * q
        rn = r @ r
        if np.sqrt(rn) <= tol * bn:
            break
        p = r + (rn / rr) * p
        rr = rn
    return P(x)


def dLdvals(A: CSR, lam: np.ndarray, V: np.ndarray, gl: np.ndarray, Gv: np.ndarray | None,
            tol: float = 1e-12) -> np.ndarray:
    """dL/dval per stored CSR entry from the N computed eigenpairs (any n)."""
    As = A.to_scipy()
    N = len(lam)
    U = V * gl[None, :]
    if Gv is not None:
        Y = np.zeros_like(V)
        for i in range(N):
            gi = Gv[:, i]
            if not np.any(gi):
                continue
            # inside the block
            c = V.T @ gi
            for j in range(N):
                if j != i and abs(lam[i] - lam[j]) > 1e-14 * max(abs(lam[i]), 1.0):
                    Y[:, i] += V[:, j] * c[j] / (lam[i] - lam[j])
            # complement: (A - lambda_i I) z = -(I - V V^T) g_i
            Y[:, i] += projected_cg(As, V, lam[i], -(gi - V @ c), tol)
        U = U + Y
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return np.einsum("ij,ij->i", U[rows], V[A.col])
