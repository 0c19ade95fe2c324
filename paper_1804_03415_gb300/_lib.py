"""ctypes binding of ``libmmdeig.so`` (argument marshalling only).

Every entry point of ``include/mmdeig.h`` is declared here with the same name.
No computation happens in Python: arrays are passed as raw pointers (numpy
host arrays or torch CUDA tensors via ``data_ptr()``).  Loading fails loudly
if the shared object is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmdeig.so")

MMD_OK, MMD_EINVAL, MMD_ENOTSPD, MMD_ENOCONV, MMD_ETIMEOUT, MMD_ECUDA, MMD_ENOMEM = 0, -1, -2, -3, -4, -5, -6
MMD_FP64, MMD_MIXED, MMD_MIXED_ALL = 0, 1, 2
MMD_HIERARCHICAL, MMD_IRLM_CG = 0, 1

i32p = C.POINTER(C.c_int32)
f64p = C.POINTER(C.c_double)


class mmd_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


class mmd_build_opts(C.Structure):
    _fields_ = [("s_max", C.c_int), ("omega_max", C.c_int), ("loc_radius", C.c_int), ("n_coarse", C.c_int),
                ("k_max", C.c_int), ("device", C.c_int), ("threads", C.c_int), ("peel", C.c_double),
                ("gpu_psi", C.c_int)]


class mmd_eig_opts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("d", C.c_int), ("c_r", C.c_int),
                ("precision", C.c_int), ("max_cg_iter", C.c_int), ("max_restarts", C.c_int),
                ("max_refine_iter", C.c_int), ("timeout_s", C.c_double), ("seed", C.c_uint64),
                ("stream", C.c_void_p), ("profile", C.c_int), ("method", C.c_int), ("stop_level", C.c_int),
                ("mg_refine", C.c_int), ("mg_op", C.c_int),
                ("poly_op", C.c_int), ("poly_refine", C.c_int), ("poly_ratio", C.c_double)]


class mmd_eig_stats(C.Structure):
    _fields_ = [("op_calls", C.c_int64), ("pcg_iters", C.c_int64), ("inner_iters", C.c_int64),
                ("b_calls", C.c_int64), ("b_iters", C.c_int64), ("refine_pcg_calls", C.c_int64),
                ("refine_pcg_iters", C.c_int64), ("restarts", C.c_int64), ("lanczos_steps", C.c_int64),
                ("refine_iters", C.c_int64), ("not_converged", C.c_int64), ("nc_solve", C.c_int64),
                ("nc_restart", C.c_int64), ("nc_refine", C.c_int64), ("kernel_launches", C.c_int64),
                ("n_levels", C.c_int), ("n_converged", C.c_int), ("norm_A", C.c_double),
                ("max_rel_residual", C.c_double), ("mu1", C.c_double), ("t_total_ms", C.c_double),
                ("pcg_launches", C.c_int64), ("pcg_ms", C.c_double), ("pcg_bytes", C.c_double),
                ("pcg_flops", C.c_double),
                ("fp64_finishes", C.c_int64), ("t_level_ms", C.c_double * 16),
                ("op0_launches", C.c_int64), ("op0_ms", C.c_double), ("op0_bytes", C.c_double),
                ("op0_flops", C.c_double), ("op0_iters", C.c_int64), ("max_pcg_iters", C.c_int64 * 16),
                ("graph_replays", C.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["t_level_ms"] = [float(v) for v in self.t_level_ms[: max(self.n_levels, 0)]]
        d["max_pcg_iters"] = [int(v) for v in self.max_pcg_iters[: max(self.n_levels, 0)]]
        return d


class mmd_level_view(C.Structure):
    _fields_ = [("n_fine", C.c_int64), ("n", C.c_int64), ("patch_of", i32p), ("patch_ptr", i32p),
                ("patch_rows", i32p), ("phi", f64p), ("omega_ptr", i32p), ("omega_rows", i32p),
                ("psi_nnz", C.c_int64), ("psi_rowptr", i32p), ("psi_col", i32p), ("psi_val", f64p),
                ("a_nnz", C.c_int64), ("a_rowptr", i32p), ("a_col", i32p), ("a_val", f64p),
                ("m_nnz", C.c_int64), ("m_rowptr", i32p), ("m_col", i32p), ("m_val", f64p),
                ("eps", C.c_double), ("delta", C.c_double), ("used_closed", C.c_int)]


SIGNATURES = {
    "mmd_default_build_opts": (None, [C.POINTER(mmd_build_opts)]),
    "mmd_default_eig_opts": (None, [C.POINTER(mmd_eig_opts)]),
    "mmd_build": (C.c_int, [C.POINTER(mmd_csr), C.POINTER(mmd_build_opts), C.POINTER(C.c_void_p)]),
    "mmd_num_levels": (C.c_int, [C.c_void_p]),
    "mmd_level_size": (C.c_int64, [C.c_void_p, C.c_int]),
    "mmd_level_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(mmd_level_view)]),
    "eig_leftmost": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(mmd_eig_opts), C.c_void_p, C.c_void_p,
                               C.c_int, C.POINTER(mmd_eig_stats)]),
    "eig_leftmost_batched": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.POINTER(mmd_eig_opts),
                                       C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "eig_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                           C.POINTER(mmd_eig_opts)]),
    "mmd_level_spmv": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mmd_level_spmv_timed": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_float), C.c_void_p]),
    "mmd_level_op": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                               C.POINTER(C.c_int64), C.c_void_p]),
    "mmd_level_op_block": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                     C.c_void_p, C.c_int, C.c_void_p]),
    "mmd_spmv_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "mmd_level_vcycle": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mmd_level_poly": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "mmd_solver_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "mmd_level_bsolve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                   C.POINTER(C.c_int64), C.c_void_p]),
    "mmd_free": (None, [C.c_void_p]),
    "mmd_strerror": (C.c_char_p, [C.c_int]),
    "mmd_last_error": (C.c_char_p, []),
    "mmd_cg_solve_noalloc": (C.c_int, [C.POINTER(mmd_csr), C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                       C.POINTER(C.c_int64), C.c_void_p]),
}

MMD_NOALLOC_MAX_N = 262144
MMD_SPMV_VARIANTS = 6
MMD_TUNE_GRIDS = 8

_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with paper_1804_03415_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MMDError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.mmd_last_error().decode()
        super().__init__(f"{where}: {lib.mmd_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def check(code, where):
    if code != MMD_OK:
        raise MMDError(code, where)
    return code
