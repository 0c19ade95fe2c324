"""The allocation-free CG entry point, checked through the C ABI against the
library's ordinary level-0 operator (mmd_level_op), which allocates its own
workspace.  Callers that may not allocate device memory during a call (fixed
memory reservations, latency-bound loops) use mmd_cg_solve_noalloc; its
working memory is a fixed array inside the library, so this file also checks
that two calls in a row (the second one reusing what the first left in the
array) give the same answers, and that sizes beyond the array are refused.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pkg():
    import paper_1804_03415_gb300 as pkg

    return pkg


def _solve_noalloc(lib, csr, b, tol, max_iter=20000):
    x = torch.zeros_like(b)
    it = C.c_int64(0)
    rc = lib.mmd_cg_solve_noalloc(C.byref(csr), b.data_ptr(), x.data_ptr(), tol, max_iter, C.byref(it), None)
    return rc, x, it.value


def test_noalloc_matches_level_op_twice():
    pkg = _pkg()
    lib = pkg._lib.load()
    A = W.fd2d(48, const=True)
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    csr = pkg._lib.mmd_csr(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=100)
    Ad = A.dense()
    cond = np.linalg.cond(Ad)
    tol = 1e-12
    rng = np.random.default_rng(2024)
    for call in range(2):
        bh = rng.standard_normal(A.n)
        b = torch.from_numpy(bh).cuda()
        rc, x, its = _solve_noalloc(lib, csr, b, tol)
        assert rc == 0, lib.mmd_last_error().decode()
        assert its > 0
        y = torch.zeros_like(b)
        h.level_op(0, b, y, tol)  # existing entry point: CG on A^(0) = A
        exact = np.linalg.solve(Ad, bh)
        bound = 10 * cond * tol * np.linalg.norm(exact)
        xn, yn = x.cpu().numpy(), y.cpu().numpy()
        assert np.linalg.norm(xn - exact) <= bound, call
        assert np.linalg.norm(xn - yn) <= 2 * bound, call
        # the residual meets the requested tolerance
        assert np.linalg.norm(bh - Ad @ xn) <= 10 * tol * np.linalg.norm(bh)
    h.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    pkg = _pkg()
    lib = pkg._lib.load()
    A = W.fd2d(8, const=True)
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    big = pkg._lib.MMD_NOALLOC_MAX_N + 1
    csr = pkg._lib.mmd_csr(big, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1)
    b = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc = lib.mmd_cg_solve_noalloc(C.byref(csr), b.data_ptr(), x.data_ptr(), 1e-8, 100, None, None)
    assert rc == pkg._lib.MMD_EINVAL
    assert b"exceeds" in lib.mmd_last_error()
