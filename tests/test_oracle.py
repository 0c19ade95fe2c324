"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

No GPU.  Every check here is independent of the oracle's own formulas:
closed-form spectra, dense LAPACK brute force, exact invariants of the
decomposition (Section 2.2-2.3, the Lemma on M^(k), Lemma 3.3) and
hand-worked partitions.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as W
from oracle import eig as E
from oracle import mmd as MM
from oracle import rng as R
from oracle import solvers as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dirichlet_closed_form(m, dim):
    k = np.arange(1, m + 1)
    s = 4.0 * np.sin(np.pi * k / (2 * (m + 1))) ** 2
    if dim == 2:
        ev = s[:, None] + s[None, :]
    else:
        ev = s[:, None, None] + s[None, :, None] + s[None, None, :]
    return np.sort(ev.ravel())


# ------------------------------------------------------------------ inputs
def test_fd_closed_form_2d_3d():
    A = W.fd2d(12, const=True)
    assert np.allclose(np.linalg.eigvalsh(A.dense()), dirichlet_closed_form(12, 2), atol=1e-12)
    B = W.fd3d(6, const=True)
    assert np.allclose(np.linalg.eigvalsh(B.dense()), dirichlet_closed_form(6, 3), atol=1e-12)


def test_workload_sizes():
    A = W.fd2d(64)
    assert (A.n, A.nnz) == (4096, 20224)
    A = W.fd3d(16)
    assert A.n == 16**3 and A.nnz == 16**3 + 6 * 16 * 16 * 15


def test_stored_large_reference_matches_the_generator():
    """The stored shift-invert reference of the torus kNN 200k workload was
    computed for the matrix the generator still produces (same integer
    pattern; values equal up to last-bit differences of exp()), a Laplacian
    plus 1e-6 I (all entries sum to 1e-6 n), and its eigenvalues are ascending,
    start at the shifted zero mode of the connected graph, and lie below the
    infinity-norm bound."""
    import hashlib

    ref = json.load(open(os.path.join(GOLDEN, "torus_knn_200k_eigs.json")))
    A = W.torus_knn(200_000, k=10, seed=W.BASE_SEED + 1)
    assert (A.n, A.nnz) == (ref["n"], ref["nnz"])
    hp = hashlib.sha256()
    for arr in (A.rowptr, A.col):
        hp.update(np.ascontiguousarray(arr).tobytes())
    assert hp.hexdigest() == ref["pattern_sha256"]
    assert abs(float(np.sum(A.val ** 2)) - ref["val_sq_sum"]) <= 1e-12 * ref["val_sq_sum"]
    assert abs(float(np.sum(A.val)) - 1e-6 * A.n) <= 1e-8
    lam = np.asarray(ref["eigenvalues"])
    assert np.all(np.diff(lam) >= 0)
    assert abs(lam[0] - 1e-6) <= 1e-12 and lam[1] > 10 * lam[0]
    assert lam[-1] <= ref["norm_A_inf"]


def test_path_graph_spectrum():
    n = 40
    ev = np.linalg.eigvalsh(W.path_graph(n).dense())
    k = np.arange(n)
    assert np.allclose(ev, np.sort(2 - 2 * np.cos(np.pi * k / n)), atol=1e-12)


# --------------------------------------------------------------------- rng
def test_splitmix64_published_vector():
    # SplitMix64 with state 0: the first outputs of the reference sequence.
    # next() = mix(state += GAMMA); our stream key for seed S, stream s is
    # mix(S + (s+1) GAMMA); with the raw mix we reproduce the sequence.
    z = R._mix(np.arange(1, 4, dtype=np.uint64) * R.GAMMA)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = R.uniform_pm1(7, 3, 1000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.1


# --------------------------------------------------------------- partition
def _csr_from_edges(n, edges):
    e = np.asarray(edges)
    return W.laplacian_from_edges(n, e[:, 0], e[:, 1], np.ones(len(e)), 1.0)


def test_partition_golden():
    cases = json.load(open(os.path.join(GOLDEN, "partition_cases.json")))["cases"]
    for c in cases:
        A = _csr_from_edges(c["n"], c["edges"])
        po, pp, pr = MM.partition(A.rowptr, A.col, A.n, c["s_max"])
        assert po.tolist() == c["patch_of"], c["name"]
        assert pp.tolist() == c["patch_ptr"], c["name"]
        assert pr.tolist() == c["patch_rows"], c["name"]


def test_neighbourhoods_golden():
    """Hand-worked psi supports (tests/golden/neighbourhood_cases.json): the
    one-ring ranking by connection count, a tie resolved to the lowest patch
    id, a patch skipped for omega_max with the next one still taken, and the
    ascending second ring."""
    g = json.load(open(os.path.join(GOLDEN, "neighbourhood_cases.json")))
    e = np.array(g["edges"])
    n = g["n"]
    A = W.laplacian_from_edges(n, e[:, 0], e[:, 1], np.ones(len(e)), 0.1).to_scipy()
    po = np.array(g["patch_of"], np.int32)
    npatch = int(po.max()) + 1
    ptr = np.zeros(npatch + 1, np.int32)
    ptr[1:] = np.cumsum(np.bincount(po))
    rows = np.lexsort((np.arange(n), po)).astype(np.int32)
    for c in g["cases"]:
        optr, orows = MM.neighbourhoods(A, po, ptr, rows, c["omega_max"], c["loc_radius"])
        got = [[int(r) for r in orows[optr[j]:optr[j + 1]]] for j in range(npatch)]
        assert got == c["omega"], c["name"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_partition_properties(seed):
    A = W.random_spd_mmatrix(300, 6.0, seed)
    po, pp, pr = MM.partition(A.rowptr, A.col, A.n, 4)
    assert sorted(pr.tolist()) == list(range(A.n))
    sizes = np.diff(pp)
    assert sizes.min() >= 1 and sizes.max() <= 8
    for j in range(len(sizes)):
        assert np.all(po[pr[pp[j]:pp[j + 1]]] == j)
        assert np.all(np.diff(pr[pp[j]:pp[j + 1]]) > 0)


# ------------------------------------------------------------ decomposition
@pytest.fixture(scope="module")
def mmd_fd():
    return MM.build(W.fd2d(24, seed=11), MM.BuildOpts(n_coarse=40))


@pytest.fixture(scope="module")
def mmd_graph():
    return MM.build(W.torus_knn(1500, seed=5), MM.BuildOpts(n_coarse=60))


@pytest.mark.parametrize("which", ["mmd_fd", "mmd_graph"])
def test_mmd_invariants(which, request):
    D = request.getfixturevalue(which)
    assert D.K >= 2
    Mprev = None
    for k, lev in enumerate(D.levels, 1):
        Phi = MM.Phi_matrix(lev).toarray()
        Psi = lev.psi.toarray()
        # Phi has orthonormal columns; Phi^T Psi = I (Section 2.2, correlation condition)
        assert np.allclose(Phi.T @ Phi, np.eye(lev.n), atol=1e-12)
        assert np.allclose(Phi.T @ Psi, np.eye(lev.n), atol=1e-10)
        # A^(k) = Psi^T A^(k-1) Psi and M^(k) = Psi^T M^(k-1) Psi, symmetric
        Aprev = D.A(k - 1).toarray()
        assert np.allclose(lev.A.toarray(), Psi.T @ Aprev @ Psi, rtol=1e-12, atol=1e-12 * abs(Aprev).max())
        Mp = np.eye(lev.n_fine) if Mprev is None else Mprev
        assert np.allclose(lev.M.toarray(), Psi.T @ Mp @ Psi, atol=1e-12)
        # lambda_min(M^(k)) >= 1 (Lemma on M^(k), Section 4)
        assert np.linalg.eigvalsh(lev.M.toarray())[0] >= 1 - 1e-10
        # lambda_min(A_st) >= lambda_min(A) (Theorem 2.2)
        assert np.linalg.eigvalsh(lev.A.toarray())[0] >= np.linalg.eigvalsh(Aprev)[0] * (1 - 1e-10)
        # Householder completion: [phi_j, U_j] orthonormal on each patch (Section 2.3)
        for j in range(0, lev.n, max(1, lev.n // 20)):
            a, b = lev.patch_ptr[j], lev.patch_ptr[j + 1]
            u = lev.uhat[a:b]
            H = np.eye(b - a) - 2 * np.outer(u, u)
            assert np.allclose(H @ H.T, np.eye(b - a), atol=1e-13)
            assert np.allclose(abs(H[:, 0]), abs(lev.phi[a:b]), atol=1e-13)
            assert np.allclose(lev.phi[a:b] @ H[:, 1:], 0, atol=1e-13)
        # U^T U = I and U^T Phi = 0 through the apply routines
        g = np.random.default_rng(k).standard_normal((lev.n_fine - lev.n, 3))
        y = MM.U_apply(lev, g)
        assert np.allclose(y.T @ y, g.T @ g, atol=1e-12)
        assert np.allclose(Phi.T @ y, 0, atol=1e-12)
        x = np.random.default_rng(k + 7).standard_normal(lev.n_fine)
        assert np.allclose(MM.Ut_apply(lev, x), (MM.U_apply(lev, np.eye(lev.n_fine - lev.n))).T @ x, atol=1e-12)
        Mprev = lev.M.toarray()


@pytest.mark.parametrize("which", ["mmd_fd", "mmd_graph"])
def test_theta_chain_monotone(which, request):
    """Lemma 3.3: A^{-1} = Theta^(0) >= Theta^(1) >= ... (so mu_i^(k) <= mu_i^(k-1))."""
    D = request.getfixturevalue(which)
    prev = 1.0 / np.linalg.eigvalsh(D.A0.toarray())  # descending mu
    for k, lev in enumerate(D.levels, 1):
        lam = sla.eigh(lev.A.toarray(), lev.M.toarray(), eigvals_only=True)
        mu = 1.0 / lam
        assert np.all(mu <= prev[:len(mu)] * (1 + 1e-9))
        prev = mu


def test_exact_psi_compression_bound():
    """Theorem 2.1 with the exact Psi = A^{-1} Phi (Phi^T A^{-1} Phi)^{-1}: ||A^{-1} - Theta|| <= eps(P)."""
    A = W.fd2d(12, seed=3)
    D = MM.build(A, MM.BuildOpts(n_coarse=10, k_max=1))
    lev = D.levels[0]
    Ad = A.dense()
    Ai = np.linalg.inv(Ad)
    Phi = MM.Phi_matrix(lev).toarray()
    Psi = Ai @ Phi @ np.linalg.inv(Phi.T @ Ai @ Phi)
    Theta = Psi @ np.linalg.inv(Psi.T @ Ad @ Psi) @ Psi.T
    assert np.linalg.norm(Ai - Theta, 2) <= lev.eps * (1 + 1e-10)
    # Theorem 2.2 upper bound: lambda_max(A_st) <= delta(P)
    assert np.linalg.eigvalsh(Psi.T @ Ad @ Psi)[-1] <= lev.delta * (1 + 1e-10)


def test_global_support_gives_the_exact_psi():
    """With Omega_j covering every patch (enough rings, no row cap) the
    constrained energy minimiser is the exact Psi = A^{-1} Phi (Phi^T A^{-1} Phi)^{-1}
    of Section 2.3 (its columns are A-orthogonal to ker Phi^T); one ring is
    not, and the exact level's smallest eigenvalue is the closest."""
    A = W.fd2d(10, const=True)
    Ad = A.dense()
    Ai = np.linalg.inv(Ad)
    lam1 = np.linalg.eigvalsh(Ad)[0]
    errs = []
    for rings in (1, 2, 50):
        D = MM.build(A, MM.BuildOpts(n_coarse=5, k_max=1, loc_radius=rings, omega_max=10**6))
        lev = D.levels[0]
        Phi = MM.Phi_matrix(lev).toarray()
        exact = Ai @ Phi @ np.linalg.inv(Phi.T @ Ai @ Phi)
        psi = lev.psi.toarray()
        if rings == 50:
            assert np.abs(psi - exact).max() <= 1e-10 * np.abs(exact).max()
        w = sla.eigh(D.A(1).toarray(), D.M(1).toarray(), eigvals_only=True)
        assert w[0] >= lam1 * (1 - 1e-12)  # Courant-Fischer: the coarse space only raises it
        errs.append(w[0] - lam1)
    assert errs[2] <= errs[1] <= errs[0]


def test_peel_bounds_eps_and_keeps_a_partition():
    """peel > 0: every patch of two or more rows ends with 1/lambda_2 <= cap
    (cap = peel x the lower median before peeling), removed rows are
    singleton patches numbered after the others, and the level still
    partitions the rows (checked against dense eigenvalues of each patch)."""
    A = W.torus_knn(1500, seed=W.BASE_SEED + 9)
    As = A.to_scipy().tocsr()
    Ad = A.dense()
    absd = np.abs(Ad)
    rowabs = absd.sum(axis=1)

    def inv_l2(S):
        AS = Ad[np.ix_(S, S)]
        E = AS - np.diag(rowabs[S] - np.abs(AS).sum(axis=1))
        w = np.linalg.eigvalsh(E)
        if w[0] < -1e-10 * np.abs(w).max():
            w = np.linalg.eigvalsh(AS)
        return 1.0 / w[1]

    po, pp, pr = MM.partition(As.indptr, As.indices, A.n, 8)
    before = sorted(inv_l2(pr[pp[j]:pp[j + 1]]) for j in range(len(pp) - 1) if pp[j + 1] - pp[j] > 1)
    cap = 3.0 * before[(len(before) - 1) // 2]
    qo, qp, qr = MM.peel(As, po, pp, pr, 3.0, 1e-10)
    npatch0 = len(pp) - 1
    assert np.array_equal(np.sort(qr), np.arange(A.n))
    assert np.array_equal(np.diff(qp)[npatch0:], np.ones(len(qp) - 1 - npatch0, dtype=np.int32))
    for j in range(len(qp) - 1):
        S = qr[qp[j]:qp[j + 1]]
        assert np.all(qo[S] == j)
        if len(S) > 1:
            assert inv_l2(S) <= cap * (1 + 1e-9)
            assert set(S) <= set(pr[pp[j]:pp[j + 1]])  # a remainder of the original patch j
    assert max(before) > cap  # the case does peel something


# ------------------------------------------------------------------ solvers
def test_cg_fpcg_bsolve():
    A = W.random_spd_mmatrix(400, 6.0, 4, shift=0.1).to_scipy()
    b = np.random.default_rng(0).standard_normal(400)
    xs = np.linalg.solve(A.toarray(), b)
    x, it, ok = S.cg(A, b, tol=1e-12)
    assert ok and np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    D = MM.build(W.random_spd_mmatrix(400, 6.0, 4, shift=0.1), MM.BuildOpts(n_coarse=20, k_max=1))
    lev = D.levels[0]
    Ak, Mk = lev.A, lev.M
    bk = np.random.default_rng(1).standard_normal(lev.n)
    x, it, ok = S.fpcg(Ak, bk, Mk, None, 1e-12)
    assert ok and np.allclose(x, np.linalg.solve(Ak.toarray(), bk), rtol=1e-8, atol=1e-10)
    y = S.op(Ak, Mk, bk, 1e-12)
    assert np.allclose(y, np.linalg.solve(Ak.toarray(), Mk @ bk), rtol=1e-8, atol=1e-10)
    U = MM.U_apply(lev, np.eye(lev.n_fine - lev.n))
    B = U.T @ A.toarray() @ U
    r = np.random.default_rng(2).standard_normal(B.shape[0])
    g = S.bsolve(A, lev, r, 1e-12)
    assert np.allclose(g, np.linalg.solve(B, r), rtol=1e-8, atol=1e-10)
    # Lemma 2.3 with kappa(U^T U) = 1: lambda_min(B) >= 1/eps(P)
    assert np.linalg.eigvalsh(B)[0] >= 1.0 / lev.eps * (1 - 1e-10)


# ------------------------------------------------------------------ Lanczos
def test_m_lanczos_arnoldi_relation_and_restart():
    """Section 4: A^{-1} M V = V T + f e^T, V^T M V = I, T symmetric tridiagonal;
    Algorithm 2 keeps the relation and the k largest Ritz values survive."""
    D = MM.build(W.fd2d(16, seed=9), MM.BuildOpts(n_coarse=20, k_max=1))
    lev = D.levels[0]
    A, M = lev.A, lev.M
    Ad, Md = A.toarray(), M.toarray()
    opf = lambda x: np.linalg.solve(Ad, Md @ x)
    Vini = np.zeros((lev.n, 0))
    lz = E.Lanczos(M, Vini, R.uniform_pm1(1, 0, lev.n), 1, 1, 1e-10)
    for _ in range(12):
        lz.step(opf)
    V, T, f = lz.V, lz.T(), lz.f
    e = np.zeros(12)
    e[-1] = 1
    rel = opf(V) - V @ T - np.outer(f, e)
    assert np.abs(rel).max() <= 1e-10 * np.abs(opf(V)).max()
    assert np.allclose(V.T @ Md @ V, np.eye(12), atol=1e-12)
    assert np.allclose(V.T @ Md @ f, 0, atol=1e-10 * np.linalg.norm(f))
    th_full = np.linalg.eigvalsh(T)
    lz.restart(8, 4)
    V, T, f = lz.V, lz.T(), lz.f
    e = np.zeros(8)
    e[-1] = 1
    rel = opf(V) - V @ T - np.outer(f, e)
    assert np.abs(rel).max() <= 1e-8 * np.abs(opf(V)).max()
    assert np.allclose(V.T @ Md @ V, np.eye(8), atol=1e-10)
    assert np.allclose(np.sort(np.linalg.eigvalsh(T)), np.sort(th_full)[4:], rtol=1e-8)


# ------------------------------------------------------------ end to end
def _check_eig(A, N, tol, opts=None, bopts=None):
    D = MM.build(A, bopts or MM.BuildOpts(n_coarse=40))
    r = E.eig_leftmost(D, N, tol, opts)
    ev, evec = np.linalg.eigh(A.dense())
    nrm = ev[-1]
    assert np.all(np.abs(r.lam - ev[:N]) <= 1e-9 * np.maximum(np.abs(ev[:N]), 1e-9 * nrm) + 1e-12 * nrm)
    res = E.residuals(A.to_scipy(), r.lam, r.V)
    assert res.max() <= 10 * tol * nrm
    assert np.allclose(r.V.T @ r.V, np.eye(N), atol=1e-8)
    return D, r


def test_eig_fd2d_small():
    _check_eig(W.fd2d(20, seed=21), 12, 1e-10)


def test_eig_const_laplacian_clusters():
    """a == 1: the Dirichlet spectrum has exact double eigenvalues (k1 <-> k2)."""
    A = W.fd2d(18, const=True)
    D, r = _check_eig(A, 10, 1e-10)
    assert np.allclose(r.lam, dirichlet_closed_form(18, 2)[:10], rtol=1e-9)


def test_eig_graph_components():
    """Shifted graph Laplacian: eigenvalue 1e-6 has multiplicity = #components."""
    A1 = W.rgg(500, deg=8.0, seed=31)
    A2 = W.rgg(400, deg=8.0, seed=32)
    n = A1.n + A2.n
    Asp = sp.block_diag([A1.to_scipy(), A2.to_scipy()]).tocsr()
    A = W.CSR(n, Asp.indptr.astype(np.int32), Asp.indices.astype(np.int32), Asp.data)
    from scipy.sparse.csgraph import connected_components
    ncomp = connected_components(Asp, directed=False)[0]
    D, r = _check_eig(A, ncomp + 4, 1e-9)
    assert np.sum(np.abs(r.lam - 1e-6) < 1e-9) == ncomp


def test_eig_level_outputs_are_top_of_each_pencil():
    """Algorithm 6: each level outputs eigenpairs of its own operator
    (A^(k))^{-1} M^(k) with the LARGEST mu (Lemma 3.2), to the level's accuracy
    eps_k (Lemma 3.3); the coarsest level keeps mu >= beta eps_K."""
    A = W.torus_knn(2500, seed=W.BASE_SEED + 40)
    D = MM.build(A, MM.BuildOpts(n_coarse=80))
    r = E.eig_leftmost(D, 20, 1e-8)
    assert D.K >= 2 and len(r.trace) == D.K + 1
    for k, mu in r.trace:
        if len(mu) == 0:
            continue
        Ak = D.A(k).toarray()
        Mk = np.eye(Ak.shape[0]) if k == 0 else D.M(k).toarray()
        top = 1.0 / sla.eigh(Ak, Mk, eigvals_only=True)[: len(mu)]
        assert np.all(np.diff(mu) <= 1e-12 * mu[0]), "descending"
        tol = 1e-8 * top[0] if k == 0 else D.levels[k - 1].eps
        assert np.abs(np.sort(mu)[::-1] - top).max() <= tol, k


# ------------------------------------------------------------------ gradient
def _loss(A, N, w, k, t):
    lam, V = np.linalg.eigh(A)
    v = V[:, k]
    return float(w @ lam[:N] + 0.5 * np.sum(t * v * v))


def test_gradient_dense_vs_finite_differences():
    """Hellmann-Feynman + first-order eigenvector perturbation against central FD."""
    from oracle import grad as OG
    Acsr = W.fd2d(6, seed=77)  # connected, simple spectrum
    A = Acsr.dense()
    N, k = 6, 1
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 1.5, N)
    t = rng.standard_normal(A.shape[0])
    lam, V = np.linalg.eigh(A)
    Gv = np.zeros((A.shape[0], N))
    Gv[:, k] = t * V[:, k]
    G = OG.dense_dLdA(A, N, w, Gv)
    h = 1e-6
    rows = np.repeat(np.arange(Acsr.n), np.diff(Acsr.rowptr))
    for e in range(0, Acsr.nnz, 7):
        r, c = rows[e], Acsr.col[e]
        E = np.zeros_like(A)
        E[r, c] = 1.0
        E[c, r] = 1.0
        fd = (_loss(A + h * E, N, w, k, t) - _loss(A - h * E, N, w, k, t)) / (2 * h)
        an = G[r, c] + (G[c, r] if r != c else 0.0)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (r, c, fd, an)


def test_gradient_block_plus_complement_matches_dense():
    """The N-pair form (in-block terms + projected CG on the complement) equals the full closed form."""
    from oracle import grad as OG
    Acsr = W.fd2d(8, seed=78)
    A = Acsr.dense()
    N, k = 8, 2
    rng = np.random.default_rng(6)
    gl = rng.uniform(0.5, 1.5, N)
    lam, V = np.linalg.eigh(A)
    t = rng.standard_normal(A.shape[0])
    Gv = np.zeros((A.shape[0], N))
    Gv[:, k] = t * V[:, k]
    Gd = OG.dense_dLdA(A, N, gl, Gv)
    rows = np.repeat(np.arange(Acsr.n), np.diff(Acsr.rowptr))
    g = OG.dLdvals(Acsr, lam[:N], V[:, :N], gl, Gv, tol=1e-13)
    assert np.allclose(g, Gd[rows, Acsr.col], atol=1e-9 * np.abs(Gd).max())
    # eigenvalue-only loss: G_rc = sum_i gl_i v_i(r) v_i(c), no solves
    g0 = OG.dLdvals(Acsr, lam[:N], V[:, :N], gl, None)
    G0 = (V[:, :N] * gl) @ V[:, :N].T
    assert np.allclose(g0, G0[rows, Acsr.col], atol=1e-13)


def test_reference_shift_invert_matches_dense():
    """The independent large-n check (shift-invert Lanczos) against dense
    LAPACK on a shifted graph Laplacian with a cluster of zero modes and on
    an FD operator."""
    from oracle import reference as RF

    for A, N in ((W.rgg(900, deg=8.0, seed=W.BASE_SEED + 90), 30), (W.fd2d(20, seed=W.BASE_SEED + 91), 25)):
        lam, V = RF.leftmost_shift_invert(A.to_scipy(), N)
        ev = np.linalg.eigvalsh(A.dense())[:N]
        assert np.abs(lam - ev).max() <= 1e-11 * np.abs(ev).max() + 1e-13 * np.abs(A.val).max()
        R = A.to_scipy() @ V - V * lam
        assert np.linalg.norm(R, axis=0).max() <= 1e-9 * np.abs(A.val).max()


def test_irlm_cg_baseline_matches_dense():
    """Section 8's baseline (implicitly restarted Lanczos on A^{-1} by plain
    CG, no decomposition) reaches the defined result: the N smallest
    eigenpairs of dense LAPACK, residual <= tol, orthonormal vectors."""
    A = W.fd2d(20, seed=W.BASE_SEED + 92)
    D = MM.build(A, MM.BuildOpts(n_coarse=40))
    r = E.eig_leftmost(D, 12, 1e-10, E.EigOpts(method="irlm_cg"))
    ev = np.linalg.eigvalsh(A.dense())
    assert np.abs(r.lam - ev[:12]).max() <= 1e-9 * np.abs(ev[:12]).max()
    assert E.residuals(A.to_scipy(), r.lam, r.V).max() <= 10 * 1e-10 * ev[-1]
    assert np.allclose(r.V.T @ r.V, np.eye(12), atol=1e-9)
    assert len(r.levels) == 1 and r.levels[0].lanczos_steps >= 12


def test_stop_level_coarse_approximation_bounds():
    """Algorithm 6 ended at level s returns Psi^(1)...Psi^(s) V^(s).  With the
    exact Psi at level 1 (supports covering every patch, Section 2.3)
    Theorem 2.1 gives ||A^{-1} - Theta^(1)|| <= eps(P^(1)), so the returned
    mu_i are within eps_1 of the true mu_i (Weyl), plus the level's Lanczos
    accuracy 0.1 eps_1 when level 1 runs an extension (s = 1 < K), and the
    residual ||A^{-1} v - mu v|| stays within 2 eps_1 (Section 7.2);
    Courant-Fischer: lambda-tilde >= lambda.  s = K is the dense solve of the
    coarsest pencil (Section 7.2), equal to LAPACK on that pencil.  The
    coefficients are random so that the spectrum has no exact multiplicity."""
    A = W.fd2d(32, seed=W.BASE_SEED + 93, log10_range=(-0.5, 0.5))
    Ad = A.dense()
    Ai = np.linalg.inv(Ad)
    ev = np.linalg.eigvalsh(Ad)
    N = 6
    for kmax, s in ((1, 1), (2, 1)):
        D = MM.build(A, MM.BuildOpts(n_coarse=12, k_max=kmax, loc_radius=50, omega_max=10**6))
        assert D.K == kmax and D.N(D.K) >= N
        eps1 = D.levels[0].eps
        r = E.eig_leftmost(D, N, 1e-10, E.EigOpts(stop_level=s))
        assert np.all(r.lam >= ev[:N] * (1 - 1e-10))
        slack = 1.0 if s == D.K else 1.1
        assert np.all(np.abs(1 / r.lam - 1 / ev[:N]) <= slack * eps1)
        assert np.linalg.norm(Ai @ r.V - r.V / r.lam, axis=0).max() <= (2.0 + slack - 1.0) * eps1
        assert np.allclose(r.V.T @ r.V, np.eye(N), atol=1e-9)
        if s == D.K:
            lamK = sla.eigh(D.A(s).toarray(), D.M(s).toarray(), eigvals_only=True)[:N]
            assert np.allclose(r.lam, lamK, rtol=1e-11)
            assert np.allclose(np.einsum("ij,ij->j", r.V, Ad @ r.V), r.lam, rtol=1e-10)


# ------------------------------------------------------------ V-cycle preconditioner
def test_chebyshev_smoother_error_polynomial():
    """The smoother's error after s steps is the scaled Chebyshev polynomial
    T_s((theta - D^{-1}A)/delta) / T_s(theta/delta) applied to the initial
    error (closed form through the eigendecomposition of D^{-1/2} A D^{-1/2})."""
    from oracle import mg as MG

    A = W.random_spd_mmatrix(60, 6.0, seed=5, shift=0.05).to_scipy()
    Ad = A.toarray()
    d = Ad.diagonal()
    hi = MG.gershgorin(A)
    lo = hi * MG.LO_FRACTION
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    w, Q = np.linalg.eigh(Ad / np.sqrt(np.outer(d, d)))
    rng = np.random.default_rng(6)
    b = rng.standard_normal(60)
    xs = np.linalg.solve(Ad, b)
    for deg in (1, 2, 3, 5):
        for x0 in (None, rng.standard_normal(60)):
            x = MG.chebyshev(A, 1.0 / d, b, x0, deg, hi)
            e0 = xs - (np.zeros(60) if x0 is None else x0)
            tpoly = np.cosh(deg * np.arccosh((theta - w) / delta + 0j)).real / np.cosh(deg * np.arccosh(theta / delta))
            # D^{-1}A = D^{-1/2} (Q w Q^T) D^{1/2}
            e_exp = (Q * tpoly) @ Q.T @ (np.sqrt(d) * e0) / np.sqrt(d)
            assert np.allclose(xs - x, e_exp, atol=1e-10 * np.abs(e0).max())
    assert hi >= w.max() * (1 - 1e-12)


def test_vcycle_coarse_correction_symmetry_and_convergence():
    """Without smoothing a one-level cycle is the Galerkin coarse solve
    Psi (Psi^T A Psi)^{-1} Psi^T r (the second term of Section 2.3's
    representation); with smoothing the cycle is a symmetric positive
    definite operator (pre and post smoothers adjoint in the A inner product);
    flexible PCG with it reaches the dense solution to tol in far fewer
    iterations than plain CG on a 1e-6-shifted graph Laplacian."""
    from oracle import mg as MG

    A = W.torus_knn(1500, seed=W.BASE_SEED + 94)
    D = MM.build(A, MM.BuildOpts(n_coarse=30, k_max=1))
    P0 = MG.VCycle(D, deg=0)
    r = np.random.default_rng(7).standard_normal(A.n)
    psi = D.levels[0].psi.toarray()
    gal = psi @ np.linalg.solve(psi.T @ A.dense() @ psi, psi.T @ r)
    assert np.allclose(P0(r), gal, atol=1e-9 * np.abs(gal).max())
    D2 = MM.build(A, MM.BuildOpts(n_coarse=30))
    assert D2.K >= 2
    P = MG.VCycle(D2, deg=2)
    Pm = P(np.eye(A.n))
    assert np.abs(Pm - Pm.T).max() <= 1e-10 * np.abs(Pm).max()
    assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T))[0] > 0
    b = np.random.default_rng(8).standard_normal(A.n)
    x, it, ok = MG.mg_pcg(A.to_scipy(), b, P, tol=1e-10)
    assert ok
    xs = np.linalg.solve(A.dense(), b)
    assert np.linalg.norm(A.to_scipy() @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    _, it_cg, _ = S.cg(A.to_scipy(), b, tol=1e-10)
    assert it * 4 < it_cg, (it, it_cg)


def test_polynomial_preconditioner_closed_form_and_pcg():
    """The level-0 polynomial preconditioner z = p(D^{-1}A) D^{-1} r equals
    (I - R(D^{-1}A)) A^{-1} r with R(t) = T_s((theta - t)/delta) / T_s(theta/delta)
    on [hi / ratio, hi] (closed form through the eigendecomposition of
    D^{-1/2} A D^{-1/2}, independent of the recurrence), is a symmetric
    positive definite operator, and flexible PCG with it reaches the dense
    solution of a 1e-6-shifted graph Laplacian to tol in fewer than a
    fifth of plain CG's iterations."""
    from oracle import mg as MG

    A = W.torus_knn(1200, seed=W.BASE_SEED + 95)
    As = A.to_scipy()
    Ad = A.dense()
    d = Ad.diagonal()
    for deg, ratio in ((1, 30.0), (4, 300.0), (16, 1000.0)):
        P = MG.PolyPrec(As, deg=deg, ratio=ratio)
        hi, lo = P.hi, P.lo
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        w, Q = np.linalg.eigh(Ad / np.sqrt(np.outer(d, d)))
        tpoly = np.cosh(deg * np.arccosh((theta - w) / delta + 0j)).real / np.cosh(deg * np.arccosh(theta / delta))
        # D^{-1}A = D^{-1/2} Q w Q^T D^{1/2}: (I - R) A^{-1} = D^{-1/2} Q ((1 - R) / w) Q^T D^{-1/2}
        Pexp = (Q * ((1.0 - tpoly) / w)) @ Q.T / np.sqrt(np.outer(d, d))
        Pm = P(np.eye(A.n))
        assert np.abs(Pm - Pexp).max() <= 1e-9 * np.abs(Pexp).max(), (deg, ratio)
        assert np.abs(Pm - Pm.T).max() <= 1e-10 * np.abs(Pm).max()
        assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T))[0] > 0
    b = np.random.default_rng(9).standard_normal(A.n)
    x, it, ok = MG.mg_pcg(As, b, MG.PolyPrec(As, deg=16, ratio=1000.0), tol=1e-10)
    assert ok
    xs = np.linalg.solve(Ad, b)
    assert np.linalg.norm(As @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    _, it_cg, _ = S.cg(As, b, tol=1e-10)
    assert it * 5 < it_cg, (it, it_cg)
