"""Oracle: linear solvers of the eigensolver's inner loop, plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``cg``    -- plain CG, the paper's pcg(A, b, -, x0, eps) (Section 4).
* ``fpcg``  -- PCG with preconditioner M whose inverse is itself applied by an
  inner CG to relative accuracy 0.1 eps (Section 4, the paragraph on solving
  M^{-1} inside PCG).  Because that inner solve is inexact the update uses the
  flexible (Polak-Ribiere) beta = z+^T (r+ - r) / (r^T z) (Golub and Ye, 1999).
* ``op``    -- Operator OP: y = pcg(A^(k), M^(k) x, M^(k), 0, eps_op) (the
  unnumbered box after Algorithm 3).
* ``bsolve`` -- g = CG(B, U^T M q) with B = U^T A U applied through the patch
  Householder reflectors (Algorithm 5, first loop; Section 2.3).

Convergence: relative residual ||b - A x||_2 <= eps ||b||_2 (the paper names
"relative error" without a norm).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import mmd as _mmd


@dataclasses.dataclass
class Counters:
    op_calls: int = 0
    pcg_iters: int = 0
    inner_iters: int = 0
    inner_calls: int = 0
    b_calls: int = 0
    b_iters: int = 0
    refine_pcg_calls: int = 0
    refine_pcg_iters: int = 0
    spmv_A: int = 0  # applications of a level stiffness matrix
    spmv_M: int = 0
    not_converged: int = 0


def cg(A, b, x0=None, tol=1e-8, maxit=100000, ctr: Counters | None = None, kind="A"):
    """Plain CG (Hestenes-Stiefel).  Returns (x, iterations, converged)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, True
    r = b - A @ x if x0 is not None else b.copy()
    rr = r @ r
    if np.sqrt(rr) <= tol * bn:
        return x, 0, True
    p = r.copy()
    for it in range(1, maxit + 1):
        q = A @ p
        if ctr is not None:
            if kind == "M":
                ctr.spmv_M += 1
            else:
                ctr.spmv_A += 1
        a = rr / (p @ q)
        x += a * p
        r -= a * q
        rr_new = r @ r
        if np.sqrt(rr_new) <= tol * bn:
            return x, it, True
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxit, False


def fpcg(A, b, M, x0=None, tol=1e-8, maxit=100000, ctr: Counters | None = None):
    """PCG with preconditioner M (M^{-1} by inner CG to 0.1 tol); M None -> plain CG."""
    if M is None:
        x, it, ok = cg(A, b, x0, tol, maxit, ctr)
        return x, it, ok
    b = np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, True
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x if x0 is not None else b.copy()
    if np.linalg.norm(r) <= tol * bn:
        return x, 0, True
    inner_tol = 0.1 * tol

    def minv(v):
        z, it, _ = cg(M, v, None, inner_tol, maxit, ctr, kind="M")
        if ctr is not None:
            ctr.inner_iters += it
            ctr.inner_calls += 1
        return z

    z = minv(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        if ctr is not None:
            ctr.spmv_A += 1
        a = rz / (p @ q)
        x += a * p
        r_new = r - a * q
        if np.linalg.norm(r_new) <= tol * bn:
            return x, it, True
        z_new = minv(r_new)
        beta = (z_new @ (r_new - r)) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r, z = r_new, z_new
    return x, maxit, False


def op(A, M, x, tol, maxit=100000, ctr: Counters | None = None):
    """Operator OP: y = pcg(A, M x, M, 0, tol); M None means M = I."""
    w = x.copy() if M is None else M @ x
    y, it, ok = fpcg(A, w, M, None, tol, maxit, ctr)
    if ctr is not None:
        ctr.op_calls += 1
        ctr.pcg_iters += it
        ctr.not_converged += 0 if ok else 1
    return y


class BOperator:
    """B = U^T A U on the complement coordinates of a level (never formed)."""

    def __init__(self, A, lev: _mmd.Level):
        self.A = A
        self.lev = lev
        n = lev.n_fine - lev.n
        self.shape = (n, n)

    def __matmul__(self, g):
        return _mmd.Ut_apply(self.lev, self.A @ _mmd.U_apply(self.lev, g))


def bsolve(A, lev: _mmd.Level, rhs, tol, maxit=100000, ctr: Counters | None = None):
    """g = CG(U^T A U, rhs, 0, tol)."""
    B = BOperator(A, lev)
    g, it, ok = cg(B, rhs, None, tol, maxit, ctr)
    if ctr is not None:
        ctr.b_calls += 1
        ctr.b_iters += it
        ctr.not_converged += 0 if ok else 1
    return g
