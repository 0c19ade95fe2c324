"""CUDA path against the CPU oracle, element by element, through the C ABI.

Tolerances (floating point, FP64 path):
  * level matrices and SpMV: 1e-12 relative (same products, different
    summation order);
  * OP / B-solve outputs: both sides stop at relative residual eps, so each
    is within cond * eps of the exact solution; they are compared with the
    exact dense solution at a tolerance derived from eps;
  * eigenvalues: relative error <= 1e-9, and eigenvectors compared as
    subspaces of clusters (relative gap < 1e-6): every principal angle
    cosine >= 1 - 1e-12 (angle <= ~1.4e-6);
  * integer level/patch indexing: bit-exact.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import eig as OE
from oracle import mmd as OM
from oracle import solvers as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pkg():
    import paper_1804_03415_gb300 as pkg

    return pkg


def _handle(A, **kw):
    pkg = _pkg()
    return pkg.MMD(A.rowptr, A.col, A.val, **kw)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def clusters(lam, rel=1e-6):
    out, cur = [], [0]
    for i in range(1, len(lam)):
        if abs(lam[i] - lam[i - 1]) <= rel * max(abs(lam[i]), abs(lam[i - 1])):
            cur.append(i)
        else:
            out.append(cur)
            cur = [i]
    out.append(cur)
    return out


def assert_eigpairs_match(lam, V, lam_ref, V_ref, rtol=1e-9, cos_tol=1e-12, lam_next=None):
    """lam_next: the (N+1)-th eigenvalue, to detect a cluster cut by N."""
    rel = np.abs(lam - lam_ref) / np.abs(lam_ref)
    assert rel.max() <= rtol, f"eigenvalue rel err {rel.max():.3e}"
    for cl in clusters(lam_ref):
        cut = cl[-1] == len(lam_ref) - 1 and lam_next is not None and \
            abs(lam_next - lam_ref[-1]) <= 1e-6 * abs(lam_next)
        if cut:
            continue  # a cluster cut by N: only the span of the whole cluster is unique
        s = np.linalg.svd(V[:, cl].T @ V_ref[:, cl], compute_uv=False)
        assert s.min() >= 1 - cos_tol, f"subspace of cluster {cl}: min cos {s.min():.16f}"


@pytest.fixture(scope="module")
def fd_case():
    A = W.fd2d(32, seed=W.BASE_SEED + 7)
    return A, OM.build(A, OM.BuildOpts(n_coarse=60))


def test_build_bitexact_and_levels(fd_case):
    A, D = fd_case
    h = _handle(A, n_coarse=60)
    assert h.num_levels == D.K
    for k in range(1, D.K + 1):
        L, O = h.level(k), D.levels[k - 1]
        for f in ["patch_of", "patch_ptr", "patch_rows", "omega_ptr", "omega_rows"]:
            assert np.array_equal(L[f], getattr(O, f)), f
        for nm, mat in [("A", O.A), ("M", O.M), ("psi", O.psi)]:
            rp, ci, va = L[nm]
            assert np.array_equal(rp, mat.indptr) and np.array_equal(ci, mat.indices), nm
            assert np.abs(va - mat.data).max() <= 1e-10 * np.abs(mat.data).max(), nm
    h.close()


def test_level_spmv(fd_case):
    A, D = fd_case
    h = _handle(A, n_coarse=60)
    rng = np.random.default_rng(1)
    for k in range(0, D.K + 1):
        n = D.N(k)
        x = rng.standard_normal(n)
        for which in ([0] if k == 0 else [0, 1]):
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            h.level_spmv(k, which, _dev(x), y)
            M = D.A(k) if which == 0 else D.M(k)
            ref = M @ x
            assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    h.close()


def test_timed_spmv_matches_plain_spmv(fd_case):
    """mmd_level_spmv_timed computes the same product as mmd_level_spmv (same
    kernel, bit-identical) and reports a positive kernel time."""
    A, D = fd_case
    h = _handle(A, n_coarse=60)
    x = np.random.default_rng(5).standard_normal(A.n)
    y1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    y2 = torch.zeros_like(y1)
    ms = h.level_spmv_timed(0, 0, _dev(x), y1, reps=3)
    h.level_spmv(0, 0, _dev(x), y2)
    assert ms > 0
    assert torch.equal(y1, y2)
    ref = A.to_scipy() @ x
    assert np.abs(y1.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    h.close()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_level_op_matches_oracle(fd_case, k):
    A, D = fd_case
    if k > D.K:
        pytest.skip("level absent")
    h = _handle(A, n_coarse=60)
    n = D.N(k)
    x = np.random.default_rng(k).standard_normal(n)
    tol = 1e-12
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    it = h.level_op(k, _dev(x), y, tol)
    ctr = OS.Counters()
    yo = OS.op(D.A(k), D.M(k), x, tol, ctr=ctr)
    Ad = D.A(k).toarray()
    rhs = x if k == 0 else D.M(k) @ x
    exact = np.linalg.solve(Ad, rhs)
    cond = np.linalg.cond(Ad)
    bound = 10 * cond * tol * np.linalg.norm(exact)
    yg = y.cpu().numpy()
    assert np.linalg.norm(yg - exact) <= bound
    assert np.linalg.norm(yo - exact) <= bound
    # same algorithm: iteration counts agree closely (rounding may move the stop by a step)
    assert abs(it - ctr.pcg_iters) <= max(2, 0.05 * ctr.pcg_iters)
    h.close()


@pytest.mark.parametrize("k,prec", [(0, 0), (1, 0), (1, 1), (0, 1), (0, 2)])
def test_level_op_block_matches_exact(fd_case, k, prec):
    """Multi-right-hand-side OP (the refinement's solver tiles): 11 columns =
    two full tiles of 4 and a ragged tile of 3, run concurrently; FP64 (prec
    0), FP32 PCG inside FP64 refinement on a coarse level (1, k = 1),
    double-float level-0 CG checked by its FP64 residual (1, k = 0) and FP32
    level-0 CG with FP64 reliable updates (2).  Each column must meet the
    same bound as the single-vector OP."""
    A, D = fd_case
    if k > D.K:
        pytest.skip("level absent")
    h = _handle(A, n_coarse=60)
    n, m, tol = D.N(k), 11, 1e-11
    X = np.random.default_rng(40 + k).standard_normal((m, n))
    Y = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    its = h.level_op_block(k, _dev(X), Y, tol, precision=prec)
    assert len(its) == m and min(its) > 0
    Ad = D.A(k).toarray()
    rhs = X.T if k == 0 else D.M(k) @ X.T
    exact = np.linalg.solve(Ad, rhs)
    cond = np.linalg.cond(Ad)
    Yg = Y.cpu().numpy().T
    for c in range(m):
        assert np.linalg.norm(Yg[:, c] - exact[:, c]) <= 10 * cond * tol * np.linalg.norm(exact[:, c]), c
    if prec == 0:  # the same iteration as the single-vector OP, column by column
        for c in (0, m - 1):
            ctr = OS.Counters()
            OS.op(D.A(k), D.M(k), X[c], tol, ctr=ctr)
            assert abs(its[c] - ctr.pcg_iters) <= max(2, 0.05 * ctr.pcg_iters)
    h.close()


@pytest.mark.parametrize("k", [1, 2])
def test_level_bsolve_matches_oracle(fd_case, k):
    A, D = fd_case
    if k > D.K:
        pytest.skip("level absent")
    h = _handle(A, n_coarse=60)
    lev = D.levels[k - 1]
    Af = D.A(k - 1)
    Mf = D.M(k - 1)
    q = np.random.default_rng(10 + k).standard_normal(lev.n_fine)
    tol = 1e-12
    x = torch.zeros(lev.n_fine, dtype=torch.float64, device="cuda")
    h.level_bsolve(k, _dev(q), x, tol)
    rhs = OM.Ut_apply(lev, q if Mf is None else Mf @ q)
    g = OS.bsolve(Af, lev, rhs, tol)
    xo = OM.U_apply(lev, g)
    U = OM.U_apply(lev, np.eye(lev.n_fine - lev.n))
    B = U.T @ Af.toarray() @ U
    exact = U @ np.linalg.solve(B, rhs)
    bound = 10 * np.linalg.cond(B) * tol * np.linalg.norm(exact)
    assert np.linalg.norm(x.cpu().numpy() - exact) <= bound
    assert np.linalg.norm(xo - exact) <= bound
    h.close()


EIG_CASES = {
    "fd2d_24": (lambda: W.fd2d(24, seed=W.BASE_SEED + 11), 16, 1e-10, 50),
    "fd2d_const_18": (lambda: W.fd2d(18, const=True), 12, 1e-10, 40),
    "torus_3000": (lambda: W.torus_knn(3000, seed=W.BASE_SEED + 12), 24, 1e-8, 80),
    "rgg_2500": (lambda: W.rgg(2500, deg=8.0, seed=W.BASE_SEED + 13), 16, 1e-8, 60),
}


_ORACLE_CACHE = {}


def _oracle_eig(name):
    """The oracle's result for an EIG_CASES entry (computed once per session)."""
    if name not in _ORACLE_CACHE:
        make, N, tol, nc = EIG_CASES[name]
        A = make()
        ref = OE.eig_leftmost(OM.build(A, OM.BuildOpts(n_coarse=nc)), N, tol)
        _ORACLE_CACHE[name] = (A, ref, np.linalg.eigvalsh(A.dense()))
    return _ORACLE_CACHE[name]


@pytest.mark.parametrize("name", sorted(EIG_CASES))
def test_eig_leftmost_matches_oracle(name):
    make, N, tol, nc = EIG_CASES[name]
    A, ref, _ = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam, V, st = h.eig_leftmost(N, tol)
    evall = _oracle_eig(name)[2]
    assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st["max_rel_residual"] <= 10 * tol
    assert np.allclose(V.T @ V, np.eye(N), atol=1e-10)
    # also against dense brute force
    ev = evall[:N]
    assert np.abs(lam - ev).max() <= 1e-9 * np.abs(ev).max() + 1e-12 * evall[-1]
    h.close()


@pytest.mark.parametrize("precision", [1, 2], ids=["mixed", "mixed_all"])
@pytest.mark.parametrize("name", ["fd2d_24", "torus_3000"])
def test_eig_leftmost_mixed_matches_oracle(name, precision):
    """MMD_MIXED (FP32 PCG on the coarse levels inside FP64 iterative
    refinement) and MMD_MIXED_ALL (level-0 CG with FP32 recurrences and FP64
    reliable updates as well) against the FP64 oracle at the FP64 path's
    tolerances: every eigenpair within 1e-9 relative, cluster subspaces
    within cos >= 1 - 1e-12, residual <= 10 tol.  The per-eigenpair errors
    are in the failure message."""
    make, N, tol, nc = EIG_CASES[name]
    A, ref, evall = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam, V, st = h.eig_leftmost(N, tol, precision=precision)
    rel = np.abs(lam - ref.lam) / np.abs(ref.lam)
    msg = "per-eigenpair relative error vs the oracle: " + " ".join(f"{x:.1e}" for x in rel)
    assert rel.max() <= 1e-9, msg
    assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st["max_rel_residual"] <= 10 * tol, st["max_rel_residual"]
    assert np.allclose(V.T @ V, np.eye(N), atol=1e-10)
    h.close()


def test_eig_device_outputs_and_edge_cases():
    pkg = _pkg()
    A = W.fd2d(12, seed=W.BASE_SEED + 14)
    h = _handle(A, n_coarse=30)
    N = 5
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    V = torch.zeros((N, A.n), dtype=torch.float64, device="cuda")
    h.eig_leftmost(N, 1e-10, out=(lam, V))
    ev = np.linalg.eigvalsh(A.dense())[:N]
    assert np.allclose(lam.cpu().numpy(), ev, rtol=1e-9)
    # N out of range, bad tol
    with pytest.raises(pkg.MMDError):
        h.eig_leftmost(0, 1e-8)
    with pytest.raises(pkg.MMDError):
        h.eig_leftmost(A.n + 1, 1e-8)
    with pytest.raises(pkg.MMDError):
        h.eig_leftmost(3, -1.0)
    h.close()
    # a matrix small enough to have no coarse level: dense solve at level 0
    B = W.fd2d(6, seed=W.BASE_SEED + 15)
    h = _handle(B, n_coarse=300)
    assert h.num_levels == 0
    lam, V, st = h.eig_leftmost(36, 1e-10)
    assert np.allclose(lam, np.linalg.eigvalsh(B.dense()), rtol=1e-9)
    h.close()


@pytest.mark.parametrize("name", ["fd2d_24", "torus_3000"])
def test_irlm_cg_baseline_matches_oracle(name):
    """MMD_IRLM_CG (Section 8's baseline: implicitly restarted Lanczos with
    plain CG, no decomposition) reaches the same defined result as the
    oracle, at the tolerances of the hierarchical path."""
    pkg = _pkg()
    make, N, tol, nc = EIG_CASES[name]
    A, ref, evall = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam, V, st = h.eig_leftmost(N, tol, method=pkg.MMD_IRLM_CG)
    assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st["max_rel_residual"] <= 10 * tol
    assert st["refine_iters"] == 0 and st["lanczos_steps"] >= N
    h.close()


def test_stop_level_matches_oracle():
    """Algorithm 6 ended at level s: s = K (dense coarsest pencil, Section
    7.2) equals the oracle's eigenpairs to 1e-10 (same pencil, same dense
    problem); s = 1 (Algorithm 6's own output V = Psi^(1) V^(1)) puts every
    mu within the level's Lanczos accuracy 0.1 eps_1 of the exact level-1
    pencil, as the oracle's does, and both lie within 1.1 eps_1 of the true
    mu (exact Psi at level 1: supports covering every patch)."""
    pkg = _pkg()
    A = W.fd2d(32, seed=W.BASE_SEED + 93, log10_range=(-0.5, 0.5))
    N = 6
    bo = dict(n_coarse=12, k_max=2, loc_radius=50, omega_max=10**6)
    D = OM.build(A, OM.BuildOpts(**bo))
    h = _handle(A, **bo)
    assert h.num_levels == D.K == 2
    ev = np.linalg.eigvalsh(A.dense())
    eps1 = D.levels[0].eps
    for s in (2, 1):
        ref = OE.eig_leftmost(D, N, 1e-10, OE.EigOpts(stop_level=s))
        lam, V, st = h.eig_leftmost(N, 1e-10, stop_level=s, allow_noconv=True)
        assert st["not_converged"] == 0
        if s == 2:
            assert np.allclose(lam, ref.lam, rtol=1e-10)
            sv = np.linalg.svd(V.T @ ref.V, compute_uv=False)
            assert sv.min() >= 1 - 1e-10
        else:
            import scipy.linalg as sla

            mu1 = 1.0 / sla.eigh(D.A(1).toarray(), D.M(1).toarray(), eigvals_only=True)[:N]
            assert np.abs(1.0 / lam - mu1).max() <= 0.1 * eps1
            assert np.abs(1.0 / ref.lam - mu1).max() <= 0.1 * eps1
            assert np.abs(1.0 / lam - 1.0 / ev[:N]).max() <= 1.1 * eps1
        assert np.allclose(V.T @ V, np.eye(N), atol=1e-9)
    with pytest.raises(pkg.MMDError):
        h.eig_leftmost(N, 1e-10, stop_level=3)
    h.close()


@pytest.mark.parametrize("m", [1, 4, 6])
def test_vcycle_matches_oracle(m):
    """One application of the level-0 V-cycle preconditioner (FP32 arithmetic
    on the device) against the oracle's FP64 V-cycle (oracle/mg.py) on the
    same levels, column by column: relative 2-norm difference <= 2e-4, the
    FP32 rounding amplified by the conditioning of the coarsest inverse
    (tiles of 1 and 4 columns and a ragged tile of 2)."""
    from oracle import mg as OMG

    A = W.torus_knn(3000, seed=W.BASE_SEED + 12)
    h = _handle(A, n_coarse=80)
    D = OM.build(A, OM.BuildOpts(n_coarse=80))
    assert D.K >= 2
    R = np.random.default_rng(40 + m).standard_normal((m, A.n))
    Z = torch.zeros((m, A.n), dtype=torch.float64, device="cuda")
    h.level_vcycle(_dev(R), Z, deg=2)
    Zo = OMG.VCycle(D, deg=2)(R.T).T
    Zg = Z.cpu().numpy()
    for c in range(m):
        err = np.linalg.norm(Zg[c] - Zo[c]) / np.linalg.norm(Zo[c])
        assert err <= 2e-4, (c, err)
    h.close()


def test_refinement_with_vcycle_matches_plain_cg():
    """The level-0 refinement preconditioned by the V-cycle (default) and by
    nothing (mg_refine = 0) give the same eigenpairs, both matching the
    oracle; the preconditioned refinement needs fewer PCG iterations."""
    name = "torus_3000"
    make, N, tol, nc = EIG_CASES[name]
    A, ref, evall = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam1, V1, st1 = h.eig_leftmost(N, tol)
    lam0, V0, st0 = h.eig_leftmost(N, tol, mg_refine=0)
    for lam, V in ((lam1, V1), (lam0, V0)):
        assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st1["refine_pcg_iters"] < st0["refine_pcg_iters"], (st1["refine_pcg_iters"], st0["refine_pcg_iters"])
    h.close()


@pytest.mark.parametrize("m", [1, 4, 6])
def test_poly_matches_oracle(m):
    """One application of the level-0 polynomial preconditioner (16 Chebyshev
    steps on [hi / 1000, hi], FP32 arithmetic on the device) against the
    oracle's FP64 one (oracle/mg.py PolyPrec), column by column: relative
    2-norm difference <= 1e-4 (FP32 rounding of each step, carried through
    the three-term recurrence); tiles of 1 and 4 columns and a ragged tile
    of 2."""
    from oracle import mg as OMG

    A = W.torus_knn(3000, seed=W.BASE_SEED + 12)
    h = _handle(A, n_coarse=80)
    R = np.random.default_rng(60 + m).standard_normal((m, A.n))
    Z = torch.zeros((m, A.n), dtype=torch.float64, device="cuda")
    h.level_poly(_dev(R), Z, deg=16, ratio=1000.0)
    Zo = OMG.PolyPrec(A.to_scipy(), deg=16, ratio=1000.0)(R.T).T
    Zg = Z.cpu().numpy()
    for c in range(m):
        err = np.linalg.norm(Zg[c] - Zo[c]) / np.linalg.norm(Zo[c])
        assert err <= 1e-4, (c, err)
    h.close()


@pytest.mark.parametrize("name", ["fd2d_24", "torus_3000"])
def test_eig_with_poly_preconditioner_matches_oracle(name):
    """Level-0 OP and refinement solves by PCG with the polynomial
    preconditioner (poly_op, poly_refine) reach the oracle's eigenpairs at
    the FP64 path's tolerances, with fewer level-0 PCG iterations than plain
    CG; so does MMD_IRLM_CG with poly_op."""
    pkg = _pkg()
    make, N, tol, nc = EIG_CASES[name]
    A, ref, evall = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam0, _, st0 = h.eig_leftmost(N, tol, mg_refine=0)
    lam, V, st = h.eig_leftmost(N, tol, poly_op=16, poly_refine=16)
    assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st["max_rel_residual"] <= 10 * tol
    assert np.allclose(V.T @ V, np.eye(N), atol=1e-10)
    assert st["pcg_iters"] < st0["pcg_iters"], (st["pcg_iters"], st0["pcg_iters"])
    lam2, V2, st2 = h.eig_leftmost(N, tol, method=pkg.MMD_IRLM_CG, poly_op=12, poly_ratio=300.0)
    assert_eigpairs_match(lam2, V2, ref.lam, ref.V, lam_next=evall[N])
    assert st2["max_rel_residual"] <= 10 * tol
    h.close()


def test_solver_tuning_picks_the_fastest_tried_grid():
    """The solver autotuner of mmd_build: on every level that runs solves
    and for both tile widths it reports the candidates it timed (resident,
    at least 64 rows per block, the smallest always tried) and the grid it
    chose is the fastest of them; the coarsest level and bad tile widths
    are refused."""
    pkg = _pkg()
    A = W.torus_knn(3000, seed=W.BASE_SEED + 12)
    h = _handle(A, n_coarse=80)
    K = h._lib.mmd_num_levels(h.h)
    assert K >= 2
    for k in range(K):
        n = h._lib.mmd_level_size(h.h, k)
        for mt in (1, 4):
            g, cand, us = h.solver_tuning(k, mt)
            tried = [(t, c) for t, c in zip(us, cand) if t > 0]
            assert tried and us[0] > 0
            assert all(c * 64 <= n or c == cand[0] for _, c in tried)
            assert g == min(tried)[1], (k, mt, g, tried)
    with pytest.raises(pkg.MMDError):
        h.solver_tuning(K, 1)
    with pytest.raises(pkg.MMDError):
        h.solver_tuning(0, 2)
    h.close()


@pytest.mark.parametrize("case,rings,peel", [("torus_4000", 1, 0.0), ("torus_4000", 2, 3.0), ("fd2d_32", 3, 0.0),
                                             ("rgg_3000", 1, 0.0)])
def test_gpu_psi_build_matches_host_build(case, rings, peel):
    """mmd_build with the local psi solves on the GPU (one block per patch,
    the default for device handles) against the host build of the same
    matrix: integer indexing bit for bit at every level, Psi, A^(k), M^(k)
    values and eps, delta to 1e-10 relative (the same local KKT systems,
    factorised in a different order)."""
    A = {"fd2d_32": lambda: W.fd2d(32, seed=3), "torus_4000": lambda: W.torus_knn(4000, seed=4),
         "rgg_3000": lambda: W.rgg(3000, seed=5)}[case]()
    om = 256 if rings == 1 else 1024
    kw = dict(n_coarse=50, peel=peel, loc_radius=rings, omega_max=om)
    hg = _handle(A, **kw)
    hh = _handle(A, device=False, **kw)
    assert hg.num_levels == hh.num_levels >= 1
    for k in range(1, hh.num_levels + 1):
        G, H = hg.level(k), hh.level(k)
        for f in ["patch_of", "patch_ptr", "patch_rows", "omega_ptr", "omega_rows"]:
            assert np.array_equal(G[f], H[f]), (k, f)
        for nm in ("A", "M", "psi"):
            assert np.array_equal(G[nm][0], H[nm][0]) and np.array_equal(G[nm][1], H[nm][1]), (k, nm)
            assert np.abs(G[nm][2] - H[nm][2]).max() <= 1e-10 * np.abs(H[nm][2]).max(), (k, nm)
        assert abs(G["eps"] - H["eps"]) <= 1e-10 * H["eps"] and abs(G["delta"] - H["delta"]) <= 1e-10 * H["delta"]
    hg.close()
    hh.close()


def test_per_level_max_pcg_counters():
    """stats.max_pcg_iters[k] (Section 7's largest iteration count of one PCG
    call on A^(k)) is at least the mean over the level-0 OP calls, at most the
    iteration cap, and zero on the dense coarsest level."""
    make, N, tol, nc = EIG_CASES["torus_3000"]
    A = make()
    h = _handle(A, n_coarse=nc)
    lam, V, st = h.eig_leftmost(N, tol, profile=1)
    mx = st["max_pcg_iters"]
    K = st["n_levels"] - 1
    assert len(mx) == K + 1 and mx[K] == 0
    assert all(0 < m <= 20000 for m in mx[:K])
    assert mx[0] * st["op0_launches"] >= st["op0_iters"] > 0
    h.close()


@pytest.mark.parametrize("name", ["torus_3000", "rgg_2500"])
def test_mixed_wide_refinement_matches_oracle(name):
    """MMD_MIXED with plain CG in the level-0 refinement (mg_refine = 0): its
    warm-started block of solves runs in the wide double-float kernel (all
    columns in one launch, FP64 residual check) and the eigenpairs match the
    oracle's at the FP64 path's tolerances."""
    make, N, tol, nc = EIG_CASES[name]
    A, ref, evall = _oracle_eig(name)
    h = _handle(A, n_coarse=nc)
    lam, V, st = h.eig_leftmost(N, tol, precision=1, mg_refine=0)
    assert_eigpairs_match(lam, V, ref.lam, ref.V, lam_next=evall[N])
    assert st["max_rel_residual"] <= 10 * tol
    assert np.allclose(V.T @ V, np.eye(N), atol=1e-10)
    h.close()


def test_wide_solve_replays_its_cuda_graph():
    """The wide multi-column launch of the MMD_MIXED refinement is recorded in
    a CUDA graph at its first call with a buffer set and replayed by the
    later refinement iterations (stats.graph_replays > 0); the eigenvalues
    agree with the FP64 path's to 1e-9 relative (absolute 1e-9 ||A||_inf for
    the 1e-6-shifted zero mode) on a 20,000-point torus kNN Laplacian, N = 100."""
    A = W.torus_knn(20000, seed=W.BASE_SEED + 21)
    h = _handle(A)
    lam64, _, st64 = h.eig_leftmost(100, 1e-8)
    lam, V, st = h.eig_leftmost(100, 1e-8, precision=1, mg_refine=0)
    assert st["graph_replays"] > 0, (st["refine_iters"], st["graph_replays"])
    assert st["n_converged"] == 100 and st["max_rel_residual"] <= 1e-8
    err = np.abs(lam - lam64)
    assert np.all(err <= np.maximum(1e-9 * np.abs(lam64), 1e-9 * st64["norm_A"])), float((err / lam64).max())
    h.close()
