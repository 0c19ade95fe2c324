"""GB300 (sm_103a) hierarchically preconditioned eigensolver (arXiv 1804.03415).

Python face of ``libmmdeig.so``; every call marshals arguments into the C ABI
declared in ``include/mmdeig.h``.  All arithmetic runs in the library's CUDA
kernels (and, for the decomposition build, its host C++); nothing here falls
back to Python or PyTorch arithmetic.

    A  = workloads.torus_knn(20000)             # any symmetric CSR
    h  = MMD(A.rowptr, A.col, A.val)            # mmd_build
    lam, V, stats = h.eig_leftmost(50, 1e-8)    # eig_leftmost
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MMD_FP64, MMD_HIERARCHICAL, MMD_IRLM_CG, MMD_MIXED, MMD_MIXED_ALL, MMDError  # noqa: F401


def build_opts(**kw) -> _lib.mmd_build_opts:
    lib = _lib.load()
    o = _lib.mmd_build_opts()
    lib.mmd_default_build_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def eig_opts(**kw) -> _lib.mmd_eig_opts:
    lib = _lib.load()
    o = _lib.mmd_eig_opts()
    lib.mmd_default_eig_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class MMD:
    """Handle of a Multiresolution Matrix Decomposition (mmd_build / mmd_free)."""

    def __init__(self, rowptr, col, val, device: bool = True, **opts):
        lib = _lib.load()
        on_dev = 0
        if hasattr(rowptr, "data_ptr"):  # torch tensors on the GPU
            on_dev = 1 if rowptr.is_cuda else 0
        if on_dev:
            n = rowptr.numel() - 1
            nnz = col.numel()
            ptrs = (rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
            self._keep = (rowptr, col, val)
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            n, nnz = len(rowptr) - 1, len(col)
            ptrs = (rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)
            self._keep = (rowptr, col, val)
        csr = _lib.mmd_csr(n, nnz, ptrs[0], ptrs[1], ptrs[2], on_dev)
        bo = build_opts(device=1 if device else 0, **opts)
        h = C.c_void_p()
        _lib.check(lib.mmd_build(C.byref(csr), C.byref(bo), C.byref(h)), "mmd_build")
        self.h = h
        self.n = n
        self.nnz = nnz
        self._lib = lib

    def close(self):
        if getattr(self, "h", None):
            self._lib.mmd_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self) -> int:
        return self._lib.mmd_num_levels(self.h)

    def level_size(self, k: int) -> int:
        return int(self._lib.mmd_level_size(self.h, k))

    def level(self, k: int) -> dict:
        """Copies of level k's arrays (natural order), 1 <= k <= K."""
        v = _lib.mmd_level_view()
        _lib.check(self._lib.mmd_level_info(self.h, k, C.byref(v)), "mmd_level_info")

        def arr(p, n, dt):
            return np.ctypeslib.as_array(p, shape=(int(n),)).astype(dt, copy=True)

        nf, n = v.n_fine, v.n
        return {
            "n_fine": nf, "n": n,
            "patch_of": arr(v.patch_of, nf, np.int32), "patch_ptr": arr(v.patch_ptr, n + 1, np.int32),
            "patch_rows": arr(v.patch_rows, nf, np.int32), "phi": arr(v.phi, nf, np.float64),
            "omega_ptr": arr(v.omega_ptr, n + 1, np.int32),
            "omega_rows": arr(v.omega_rows, arr(v.omega_ptr, n + 1, np.int32)[-1], np.int32),
            "psi": (arr(v.psi_rowptr, nf + 1, np.int32), arr(v.psi_col, v.psi_nnz, np.int32),
                    arr(v.psi_val, v.psi_nnz, np.float64)),
            "A": (arr(v.a_rowptr, n + 1, np.int32), arr(v.a_col, v.a_nnz, np.int32), arr(v.a_val, v.a_nnz, np.float64)),
            "M": (arr(v.m_rowptr, n + 1, np.int32), arr(v.m_col, v.m_nnz, np.int32), arr(v.m_val, v.m_nnz, np.float64)),
            "eps": v.eps, "delta": v.delta, "used_closed": v.used_closed,
        }

    # ---- level operators on CUDA tensors (torch) in natural order
    def level_spmv(self, k, which, x, y, stream=0):
        _lib.check(self._lib.mmd_level_spmv(self.h, k, which, x.data_ptr(), y.data_ptr(), stream), "mmd_level_spmv")

    def level_spmv_timed(self, k, which, x, y, reps=20, stream=0) -> float:
        """y = A^(k) x (or M^(k) x) computed reps times; returns ms per SpMV kernel."""
        ms = C.c_float(0.0)
        _lib.check(self._lib.mmd_level_spmv_timed(self.h, k, which, x.data_ptr(), y.data_ptr(), reps, C.byref(ms),
                                                  stream), "mmd_level_spmv_timed")
        return float(ms.value)

    def level_op(self, k, x, y, tol, max_iter=20000, stream=0) -> int:
        it = C.c_int64(0)
        _lib.check(self._lib.mmd_level_op(self.h, k, x.data_ptr(), y.data_ptr(), tol, max_iter, C.byref(it), stream),
                   "mmd_level_op")
        return it.value

    def level_op_block(self, k, X, Y, tol, max_iter=20000, precision=MMD_FP64, stream=0):
        """Y = OP(X) column by column; X, Y: CUDA float64 tensors (m, n_k), one row per column."""
        m = X.shape[0]
        its = (C.c_int64 * m)()
        _lib.check(self._lib.mmd_level_op_block(self.h, k, m, X.data_ptr(), Y.data_ptr(), tol, max_iter, its,
                                                precision, stream), "mmd_level_op_block")
        return list(its)

    def spmv_tuning(self, k=0, which=0):
        """(chosen single-column SpMV variant, ms of every variant) of A^(k) / M^(k)."""
        ms = (C.c_float * _lib.MMD_SPMV_VARIANTS)()
        v = self._lib.mmd_spmv_tuning(self.h, k, which, ms)
        if v < 0:
            _lib.check(v, "mmd_spmv_tuning")
        return v, [float(x) for x in ms]

    def solver_tuning(self, k=0, mt=1):
        """(chosen solver grid, candidate grids, us per CG iteration of every
        candidate, 0 = not tried) of level k for tiles of mt columns."""
        g = (C.c_int * _lib.MMD_TUNE_GRIDS)()
        us = (C.c_float * _lib.MMD_TUNE_GRIDS)()
        v = self._lib.mmd_solver_tuning(self.h, k, mt, g, us)
        if v < 0:
            _lib.check(v, "mmd_solver_tuning")
        return v, [int(x) for x in g], [float(x) for x in us]

    def level_vcycle(self, R, Z, deg=2, stream=0):
        """Z = V(R): one application of the level-0 V-cycle preconditioner;
        R, Z: CUDA float64 tensors (m, n), one row per column."""
        _lib.check(self._lib.mmd_level_vcycle(self.h, R.shape[0], R.data_ptr(), Z.data_ptr(), deg, stream),
                   "mmd_level_vcycle")

    def level_poly(self, R, Z, deg=16, ratio=1000.0, stream=0):
        """Z = p(D^{-1}A) D^{-1} R: one application of the level-0 polynomial
        preconditioner; R, Z: CUDA float64 tensors (m, n), one row per column."""
        _lib.check(self._lib.mmd_level_poly(self.h, R.shape[0], R.data_ptr(), Z.data_ptr(), deg, ratio, stream),
                   "mmd_level_poly")

    def level_bsolve(self, k, q, x, tol, max_iter=20000, stream=0) -> int:
        it = C.c_int64(0)
        _lib.check(self._lib.mmd_level_bsolve(self.h, k, q.data_ptr(), x.data_ptr(), tol, max_iter, C.byref(it),
                                              stream), "mmd_level_bsolve")
        return it.value

    def eig_leftmost(self, N: int, tol: float, out=None, allow_noconv: bool = False, **opts):
        """N smallest eigenpairs.  ``out``: None (host numpy) or (lam, V) CUDA tensors."""
        o = eig_opts(**opts)
        st = _lib.mmd_eig_stats()
        if out is None:
            lam = np.zeros(N)
            V = np.zeros((N, self.n))  # column-major n x N == row-major N x n
            rc = self._lib.eig_leftmost(self.h, N, tol, C.byref(o), lam.ctypes.data, V.ctypes.data, 0, C.byref(st))
            res = (lam, V.T)
        else:
            lam_t, V_t = out
            rc = self._lib.eig_leftmost(self.h, N, tol, C.byref(o), lam_t.data_ptr(), V_t.data_ptr(), 1, C.byref(st))
            res = (lam_t, V_t)
        if rc != _lib.MMD_OK and not (allow_noconv and rc == _lib.MMD_ENOCONV):
            _lib.check(rc, "eig_leftmost")
        return res[0], res[1], st.as_dict()

    def eig_grad(self, dL_dlambda, dL_dV=None, out=None, **opts):
        """dL/dval per stored CSR entry for the last eig_leftmost result.

        Host numpy inputs -> host numpy output; CUDA tensors -> CUDA tensor
        (or ``out``)."""
        o = eig_opts(**opts)
        if hasattr(dL_dlambda, "data_ptr"):
            import torch

            g = out if out is not None else torch.zeros(self.nnz, dtype=torch.float64, device=dL_dlambda.device)
            gv = dL_dV.contiguous() if dL_dV is not None else None
            rc = self._lib.eig_grad(self.h, dL_dlambda.data_ptr(), gv.data_ptr() if gv is not None else None, 1,
                                    g.data_ptr(), 1, C.byref(o))
            _lib.check(rc, "eig_grad")
            return g
        gl = np.ascontiguousarray(dL_dlambda, dtype=np.float64)
        g = np.zeros(self.nnz)
        gv = None
        if dL_dV is not None:
            gv = np.ascontiguousarray(np.asarray(dL_dV, dtype=np.float64).T)  # (N, n) rows = columns of n x N
        rc = self._lib.eig_grad(self.h, gl.ctypes.data, gv.ctypes.data if gv is not None else None, 0,
                                g.ctypes.data, 0, C.byref(o))
        _lib.check(rc, "eig_grad")
        return g


def eig_leftmost_batched(handles, N, tol: float, streams: int = 8, allow_noconv: bool = False, **opts):
    """N[i] smallest eigenpairs of each handle's matrix, the problems solved
    concurrently on ``streams`` CUDA streams (eig_leftmost_batched).

    ``N``: int or one int per handle.  Returns lists (lam_i, V_i, stats_i),
    host numpy arrays.  With ``allow_noconv`` an iteration cap in some problem
    returns the best pairs found (stats_i["n_converged"] tells which)."""
    lib = _lib.load()
    cnt = len(handles)
    Ns = [int(N)] * cnt if np.isscalar(N) else [int(x) for x in N]
    if len(Ns) != cnt:
        raise ValueError("one N per handle")
    o = eig_opts(**opts)
    lams = [np.zeros(Ns[i]) for i in range(cnt)]
    Vs = [np.zeros((Ns[i], handles[i].n)) for i in range(cnt)]
    hs = (C.c_void_p * cnt)(*[h.h.value for h in handles])
    na = (C.c_int * cnt)(*Ns)
    lp = (C.c_void_p * cnt)(*[a.ctypes.data for a in lams])
    vp = (C.c_void_p * cnt)(*[a.ctypes.data for a in Vs])
    st = (_lib.mmd_eig_stats * cnt)()
    rc = lib.eig_leftmost_batched(hs, cnt, na, tol, C.byref(o), lp, vp, 0, st, streams)
    if rc != _lib.MMD_OK and not (allow_noconv and rc == _lib.MMD_ENOCONV):
        _lib.check(rc, "eig_leftmost_batched")
    return [(lams[i], Vs[i].T, st[i].as_dict()) for i in range(cnt)]


def eigsh_leftmost(rowptr, col, val, N: int, tol: float = 1e-8, build=None, **opts):
    """Differentiable leftmost eigenpairs of the symmetric CSR matrix (rowptr, col, val).

    ``val`` is a CUDA float64 tensor (the values that receive gradients);
    rowptr / col are int32 tensors.  Returns (lambda (N,), V (n, N)).  The
    forward pass is eig_leftmost, the backward pass eig_grad.
    """
    import torch

    class _Eig(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v):
            h = MMD(rowptr, col, v, **(build or {}))
            n = rowptr.numel() - 1
            lam = torch.zeros(N, dtype=torch.float64, device=v.device)
            Vt = torch.zeros((N, n), dtype=torch.float64, device=v.device)
            h.eig_leftmost(N, tol, out=(lam, Vt), **opts)
            ctx.h = h
            return lam, Vt.T

        @staticmethod
        def backward(ctx, glam, gV):
            # the handle keeps the forward result, so backward may run more than
            # once (retain_graph); it is freed with the graph (MMD.__del__)
            gl = glam if glam is not None else torch.zeros(N, dtype=torch.float64, device=val.device)
            gv = gV.T.contiguous() if gV is not None else None
            return ctx.h.eig_grad(gl.contiguous(), gv)

    return _Eig.apply(val)
