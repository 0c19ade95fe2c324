"""eig_grad (adjoint of the eigensolver) against the CPU oracle's gradient and
against central finite differences of the loss.

Loss: L = sum_{i<N} w_i lambda_i + 1/2 sum_j t_j v_k(j)^2 (sign-invariant in
v_k), so dL/dlambda = w and dL/dV has one nonzero column t * v_k.  The oracle
computes its own eigenpairs (dense LAPACK) and its own gradient; only the
loss definition is shared.  Tolerance: relative 1e-6 of the largest entry
(both sides stop their eigensolves and adjoint solves at ~1e-10..1e-12).
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(A, N, k, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, N)
    t = rng.standard_normal(A.n)
    return w, t


def test_eig_grad_matches_oracle_fd2d():
    import paper_1804_03415_gb300 as pkg

    A = W.fd2d(16, seed=W.BASE_SEED + 31)
    N, k = 8, 1
    w, t = _setup(A, N, k, 3)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=40)
    lam, V, st = h.eig_leftmost(N, 1e-11)
    Gv = np.zeros((A.n, N))
    Gv[:, k] = t * V[:, k]
    g = h.eig_grad(w, Gv)
    # oracle: its own eigenpairs and gradient
    lo, Vo = np.linalg.eigh(A.dense())
    Gvo = np.zeros((A.n, N))
    Gvo[:, k] = t * Vo[:, k]
    go = OG.dLdvals(A, lo[:N], Vo[:, :N], w, Gvo, tol=1e-13)
    assert np.abs(g - go).max() <= 1e-6 * np.abs(go).max()
    # eigenvalue-only loss (no adjoint solve)
    g0 = h.eig_grad(w, None)
    go0 = OG.dLdvals(A, lo[:N], Vo[:, :N], w, None)
    assert np.abs(g0 - go0).max() <= 1e-8 * np.abs(go0).max()
    h.close()


def test_eig_grad_finite_differences_rgg():
    import paper_1804_03415_gb300 as pkg

    A = W.rgg(600, deg=10.0, seed=W.BASE_SEED + 32, weights=(0.5, 2.0), lcc=True)
    N, k = 10, 1
    w, t = _setup(A, N, k, 4)

    def loss(vals):
        h = pkg.MMD(A.rowptr, A.col, vals, n_coarse=60)
        lam, V, _ = h.eig_leftmost(N, 1e-12)
        h.close()
        return float(w @ lam + 0.5 * np.sum(t * V[:, k] ** 2))

    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=60)
    lam, V, _ = h.eig_leftmost(N, 1e-12)
    Gv = np.zeros((A.n, N))
    Gv[:, k] = t * V[:, k]
    g = h.eig_grad(w, Gv)
    h.close()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    rng = np.random.default_rng(9)
    off = np.where(rows < A.col)[0]
    hstep = 1e-6
    for e in rng.choice(off, size=6, replace=False):
        r, c = rows[e], A.col[e]
        e2 = A.rowptr[c] + np.searchsorted(A.col[A.rowptr[c]:A.rowptr[c + 1]], r)
        vp, vm = A.val.copy(), A.val.copy()
        vp[e] += hstep
        vp[e2] += hstep
        vm[e] -= hstep
        vm[e2] -= hstep
        fd = (loss(vp) - loss(vm)) / (2 * hstep)
        an = g[e] + g[e2]
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (r, c, fd, an)


def test_autograd_function():
    import paper_1804_03415_gb300 as pkg

    A = W.fd2d(12, seed=W.BASE_SEED + 33)
    N = 5
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda().requires_grad_(True)
    lam, V = pkg.eigsh_leftmost(rp, ci, va, N, 1e-11, build={"n_coarse": 30})
    lam.sum().backward()
    lo, Vo = np.linalg.eigh(A.dense())
    go = OG.dLdvals(A, lo[:N], Vo[:, :N], np.ones(N), None)
    assert np.abs(va.grad.cpu().numpy() - go).max() <= 1e-8 * np.abs(go).max()


def test_autograd_eigenvector_only_loss_and_second_backward():
    """A loss that uses V alone (dL/dlambda undefined) goes through backward,
    matches the oracle's gradient, and a second backward on the retained
    graph gives the same gradient again."""
    import paper_1804_03415_gb300 as pkg

    A = W.fd2d(12, seed=W.BASE_SEED + 34)
    N, k = 5, 1
    t = np.random.default_rng(5).standard_normal(A.n)
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda().requires_grad_(True)
    lam, V = pkg.eigsh_leftmost(rp, ci, va, N, 1e-12, build={"n_coarse": 30})
    tt = torch.from_numpy(t).cuda()
    loss = 0.5 * (tt * V[:, k] ** 2).sum()
    loss.backward(retain_graph=True)
    g1 = va.grad.detach().clone()
    lo, Vo = np.linalg.eigh(A.dense())
    Gvo = np.zeros((A.n, N))
    Gvo[:, k] = t * Vo[:, k]
    go = OG.dLdvals(A, lo[:N], Vo[:, :N], np.zeros(N), Gvo, tol=1e-13)
    assert np.abs(g1.cpu().numpy() - go).max() <= 1e-6 * np.abs(go).max()
    va.grad = None
    loss.backward()
    assert torch.allclose(va.grad, g1, rtol=0, atol=1e-12 * float(g1.abs().max()))
