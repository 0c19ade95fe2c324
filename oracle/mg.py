"""Oracle: the decomposition's levels applied as a V-cycle preconditioner (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2.3 writes A^{-1} = U B^{-1} U^T + Psi (Psi^T A Psi)^{-1} Psi^T (the
representation behind the MMD, exact for the exact Psi, with B = U^T A U
bounded by Lemma 2.3), and its K-level form.  With localized Psi the
representation is no longer exact, so the library uses it as a preconditioner
of the warm-started level-0 solves of the refinement (Algorithm 5; its
right-hand sides are not restricted to an invariant subspace, the situation
in which Section 4 prefers plain CG).  The two terms are applied one after
the other, level by level, as a symmetric V-cycle:

* the fine-scale part (range U, well conditioned) by a Chebyshev polynomial
  smoother of D^{-1} A^(k) (D = diag A^(k)) of degree s on the interval
  [hi / 30, hi], hi = the Gershgorin bound max_i sum_j |a_ij| / a_ii of
  D^{-1} A^(k) (s steps before and s after the coarse correction);
* the coarse part by restriction Psi^(k+1)^T of the residual, the same
  cycle on A^(k+1), and prolongation Psi^(k+1);
* the coarsest level by a dense solve with A^(K).

The outer iteration is the flexible PCG of ``solvers.fpcg`` with this
preconditioner; its result is A^{-1} b to the same relative residual as
plain CG, so the refinement's output is unchanged.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mmd as _mmd

LO_FRACTION = 1.0 / 30.0


def gershgorin(A: sp.spmatrix) -> float:
    """max_i sum_j |a_ij| / a_ii: an upper bound of lambda_max(D^{-1} A)."""
    A = sp.csr_matrix(A)
    return float((np.asarray(abs(A).sum(axis=1)).ravel() / A.diagonal()).max())


def chebyshev(A, dinv, b, x0, deg: int, hi: float, lo: float | None = None):
    """deg steps of Chebyshev iteration for A x = b preconditioned by D^{-1},
    eigenvalue interval [lo, hi], lo = hi * LO_FRACTION unless given (x0 None
    means x0 = 0).

    theta = (hi + lo) / 2, delta = (hi - lo) / 2, sigma = theta / delta;
    d_0 = D^{-1}(b - A x_0) / theta;  rho_0 = 1 / sigma;
    rho_k = 1 / (2 sigma - rho_{k-1}),
    d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^{-1}(b - A x_k);
    x_{k+1} = x_k + d_k.  The error obeys e_deg = T_deg((theta - D^{-1}A)/delta)
    / T_deg(sigma) e_0 (T the Chebyshev polynomial of the first kind)."""
    if lo is None:
        lo = hi * LO_FRACTION
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if deg <= 0:
        return x
    res = b - A @ x if x0 is not None else b
    d = dinv * res / theta
    x = x + d
    rho = 1.0 / sigma
    for _ in range(1, deg):
        rho_new = 1.0 / (2.0 * sigma - rho)
        res = b - A @ x
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * res)
        x = x + d
        rho = rho_new
    return x


class VCycle:
    """The V-cycle preconditioner on the levels of a decomposition (Algorithm 6's
    levels 0..K: A^(k), Psi^(k+1)); ``deg`` Chebyshev steps per smoothing."""

    def __init__(self, D: _mmd.MMD, deg: int = 2):
        self.deg = deg
        self.K = D.K
        self.A = [sp.csr_matrix(D.A(k)) for k in range(D.K + 1)]
        self.dinv = [1.0 / self.A[k].diagonal() for k in range(D.K)]
        self.hi = [gershgorin(self.A[k]) for k in range(D.K)]
        self.psi = [sp.csr_matrix(lev.psi) for lev in D.levels]
        self.coarse = self.A[D.K].toarray()

    def cycle(self, r, k: int = 0):
        if k == self.K:
            return np.linalg.solve(self.coarse, r)
        A, dinv, hi = self.A[k], self.dinv[k], self.hi[k]
        x = chebyshev(A, dinv, r, None, self.deg, hi)
        rc = self.psi[k].T @ (r - A @ x)
        x = x + self.psi[k] @ self.cycle(rc, k + 1)
        return chebyshev(A, dinv, r, x, self.deg, hi)

    def __call__(self, r):
        r = np.asarray(r, dtype=np.float64)
        if r.ndim == 1:
            return self.cycle(r)
        return np.stack([self.cycle(r[:, c]) for c in range(r.shape[1])], axis=1)


class PolyPrec:
    """The polynomial preconditioner of the level-0 solves:
    z = p(D^{-1}A) D^{-1} r, ``deg`` steps of ``chebyshev`` for A z = r from
    z = 0 on the interval [hi / ratio, hi] of D^{-1} A.  Not in the paper
    (its level 0 is not computed, and Operator OP there is PCG with M^(k),
    which is the identity at level 0); it changes how A^{-1} b is reached,
    not its value.  With the residual polynomial R(t) = T_deg((theta - t) /
    delta) / T_deg(theta / delta) of the interval, the operator is
    (I - R(D^{-1}A)) A^{-1}: symmetric, and positive definite when
    |R| < 1 on the spectrum of D^{-1} A, which holds on (0, hi]."""

    def __init__(self, A, deg: int = 16, ratio: float = 1000.0):
        self.A = sp.csr_matrix(A)
        self.deg = deg
        self.dinv = 1.0 / self.A.diagonal()
        self.hi = gershgorin(self.A)
        self.lo = self.hi / ratio

    def __call__(self, r):
        r = np.asarray(r, dtype=np.float64)
        if r.ndim == 1:
            return chebyshev(self.A, self.dinv, r, None, self.deg, self.hi, self.lo)
        return np.stack([chebyshev(self.A, self.dinv, r[:, c], None, self.deg, self.hi, self.lo)
                         for c in range(r.shape[1])], axis=1)


def mg_pcg(A, b, P, x0=None, tol=1e-8, maxit=100000):
    """Flexible PCG (the update of solvers.fpcg) with z = P(r).
    Returns (x, iterations, converged)."""
    b = np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, True
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x if x0 is not None else b.copy()
    if np.linalg.norm(r) <= tol * bn:
        return x, 0, True
    z = P(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r_new = r - a * q
        if np.linalg.norm(r_new) <= tol * bn:
            return x, it, True
        z_new = P(r_new)
        beta = (z_new @ (r_new - r)) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r = r_new
    return x, maxit, False
