"""C ABI on the CPU: the library loads, exports every declared entry point,
and its host-only decomposition build is bit-exact with the oracle's integer
indexing (patches, supports, symbolic patterns) and matches its floats."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import mmd as OM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1804_03415_gb300 import build as B

    B.build()
    import paper_1804_03415_gb300 as P

    P._lib.load()
    return P


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mmdeig.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+\**\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(pkg):
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(pkg._lib.LIB_PATH)
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) <= set(pkg._lib.SIGNATURES), set(names) - set(pkg._lib.SIGNATURES)


def test_strerror_and_validation(pkg):
    lib = pkg._lib.load()
    assert lib.mmd_strerror(0) == b"ok"
    assert lib.mmd_strerror(-3).startswith(b"iteration")
    # malformed CSR: unsorted columns, asymmetric values, missing diagonal
    A = W.fd2d(4, const=True)
    bad = A.col.copy()
    bad[[1, 2]] = bad[[2, 1]]
    with pytest.raises(pkg.MMDError):
        pkg.MMD(A.rowptr, bad, A.val, device=False)
    v = A.val.copy()
    v[1] += 0.5
    with pytest.raises(pkg.MMDError):
        pkg.MMD(A.rowptr, A.col, v, device=False)
    # a row without its diagonal
    rp, ci, va = A.rowptr.copy(), A.col.copy(), A.val.copy()
    i0 = np.where(ci[rp[0]:rp[1]] == 0)[0][0]
    keep = np.ones(len(ci), bool)
    keep[rp[0] + i0] = False
    rp2 = rp.copy()
    rp2[1:] -= 1
    with pytest.raises(pkg.MMDError):
        pkg.MMD(rp2, ci[keep], va[keep], device=False)


@pytest.mark.parametrize("case,peel,rings", [("fd2d_32", 0.0, 1), ("torus_4000", 0.0, 1), ("rgg_3000", 0.0, 1),
                                             ("torus_4000", 3.0, 2), ("fd2d_32", 2.0, 3)])
def test_host_build_matches_oracle(pkg, case, peel, rings):
    """Library build vs oracle build: integer indexing bit-exact, values to
    1e-10; also with eps-bounded patches (peel) and wider psi supports."""
    A = {"fd2d_32": lambda: W.fd2d(32, seed=3), "torus_4000": lambda: W.torus_knn(4000, seed=4),
         "rgg_3000": lambda: W.rgg(3000, seed=5)}[case]()
    om = 256 if rings == 1 else 1024
    h = pkg.MMD(A.rowptr, A.col, A.val, device=False, n_coarse=50, peel=peel, loc_radius=rings, omega_max=om)
    D = OM.build(A, OM.BuildOpts(n_coarse=50, peel=peel, loc_radius=rings, omega_max=om))
    assert h.num_levels == D.K
    for k in range(1, D.K + 1):
        L, O = h.level(k), D.levels[k - 1]
        for f in ["patch_of", "patch_ptr", "patch_rows", "omega_ptr", "omega_rows"]:
            assert np.array_equal(L[f], getattr(O, f)), (k, f)
        for nm, mat in [("A", O.A), ("M", O.M), ("psi", O.psi)]:
            rp, ci, va = L[nm]
            assert np.array_equal(rp, mat.indptr) and np.array_equal(ci, mat.indices), (k, nm)
            assert np.abs(va - mat.data).max() <= 1e-10 * np.abs(mat.data).max(), (k, nm)
        assert abs(L["eps"] - O.eps) <= 1e-10 * O.eps
        assert abs(L["delta"] - O.delta) <= 1e-10 * O.delta
        assert L["used_closed"] == O.used_closed
    h.close()


def test_entry_points_refuse_host_only_handles_and_bad_options(pkg):
    """Calls that need the device levels refuse a host-only handle with
    MMD_EINVAL (and a message) before touching any device memory; build
    options out of range are refused too.  No GPU is used."""
    import ctypes as C

    lib = pkg._lib.load()
    A = W.fd2d(8, seed=11)
    h = pkg.MMD(A.rowptr, A.col, A.val, device=False, n_coarse=20)
    lam = np.zeros(3)
    V = np.zeros((3, A.n))
    st = pkg._lib.mmd_eig_stats()
    o = pkg.eig_opts()
    assert lib.eig_leftmost(h.h, 3, 1e-8, C.byref(o), lam.ctypes.data, V.ctypes.data, 0, C.byref(st)) == \
        pkg._lib.MMD_EINVAL
    hs = (C.c_void_p * 1)(h.h.value)
    na = (C.c_int * 1)(3)
    lp = (C.c_void_p * 1)(lam.ctypes.data)
    vp = (C.c_void_p * 1)(V.ctypes.data)
    assert lib.eig_leftmost_batched(hs, 1, na, 1e-8, C.byref(o), lp, vp, 0, None, 2) == pkg._lib.MMD_EINVAL
    assert b"problem 0" in lib.mmd_last_error()
    its = (C.c_int64 * 2)()
    assert lib.mmd_level_op_block(h.h, 0, 2, V.ctypes.data, V.ctypes.data, 1e-8, 10, its, 0, None) == \
        pkg._lib.MMD_EINVAL
    g = np.zeros(A.nnz)
    assert lib.eig_grad(h.h, lam.ctypes.data, None, 0, g.ctypes.data, 0, C.byref(o)) == pkg._lib.MMD_EINVAL
    assert lib.mmd_solver_tuning(h.h, 0, 1, None, None) == pkg._lib.MMD_EINVAL
    h.close()
    for bad in ({"peel": -1.0}, {"loc_radius": -1}, {"s_max": 0}):
        with pytest.raises(pkg.MMDError):
            pkg.MMD(A.rowptr, A.col, A.val, device=False, **bad)


def test_build_refuses_nonfinite_and_non_spd_inputs(pkg):
    """Failure paths of mmd_build made on the host: NaN / Inf values ->
    MMD_EINVAL; a non-positive diagonal, or a positive diagonal whose patch
    matrix is indefinite -> MMD_ENOTSPD.  Nothing reaches a GPU."""
    lib = pkg._lib
    A = W.fd2d(6, seed=W.BASE_SEED + 60)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = np.where(rows != A.col)[0]
    for bad in (np.nan, np.inf, -np.inf):
        v = A.val.copy()
        e = off[3]
        r, c = rows[e], A.col[e]
        e2 = A.rowptr[c] + np.searchsorted(A.col[A.rowptr[c]:A.rowptr[c + 1]], r)
        v[e] = v[e2] = bad
        with pytest.raises(pkg.MMDError) as ei:
            pkg.MMD(A.rowptr, A.col, v, device=False)
        assert ei.value.code == lib.MMD_EINVAL
    v = A.val.copy()
    d = A.rowptr[5] + np.searchsorted(A.col[A.rowptr[5]:A.rowptr[6]], 5)
    v[d] = -1.0
    with pytest.raises(pkg.MMDError) as ei:
        pkg.MMD(A.rowptr, A.col, v, device=False)
    assert ei.value.code == lib.MMD_ENOTSPD
    # I + 2 x (path adjacency): positive diagonal, eigenvalues 1 + 4 cos(pi k / 9) < 0 for some k
    n = 8
    i = np.arange(n - 1)
    P = W.laplacian_from_edges(n, i, i + 1, -2.0 * np.ones(n - 1), 0.0)  # D - W with W = -2
    val = P.val.copy()
    rr = np.repeat(np.arange(n), np.diff(P.rowptr))
    val[rr == P.col] = 1.0
    with pytest.raises(pkg.MMDError) as ei:
        pkg.MMD(P.rowptr, P.col, val, device=False, n_coarse=2)
    assert ei.value.code == lib.MMD_ENOTSPD
