"""Oracle: Multiresolution Matrix Decomposition (MMD) build, plain FP64.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package; the library never
does.  It shares no code with the CUDA path.

The paper (Section 2.2-2.3) builds the decomposition with an adaptive
partitioner from an earlier paper that is not part of this one.  What the
method needs from a level is fixed by the paper; how the patches are chosen
is not.  This file implements one fixed, integer-only construction so that the
library's own (separate) build can be compared with it bit for bit:

Per level k (input matrix A = A^(k-1) of size n, with M^(0) = I):

1. Partition the pattern of A (diagonal excluded) into patches P_j
   (aggregation, ``partition``).  Integer-only.
2. phi_j = normalised eigenvector of the smallest eigenvalue of the patch's
   interior energy  A[S,S] - diag(sum_{j not in S} |a_ij|)  (Section 2.2,
   q = 1); if that matrix is not PSD the closed energy A[S,S] is used.
   Sign: largest-|.| entry positive (ties: lowest position).
3. Error factor eps(P) = max_j 1/lambda_2(patch energy) (Section 2.2) and
   condition factor delta(P) = max_j 1/(phi_j^T A[S,S]^{-1} phi_j)
   (Theorem 2.2).
4. Householder vector u_j = phi_j + sign(phi_j[0]) e_0, stored normalised;
   H_j = I - 2 u u^T, U_j = columns 1.. of H_j (Section 2.3, orthonormal
   completion of phi_j so that kappa(U^T U) = 1).
5. Localised psi_j: psi_j = argmin psi^T A psi subject to phi_i^T psi = delta_ij
   for every patch i inside Omega_j and supp psi in Omega_j, where Omega_j is
   P_j plus whole neighbouring patches (the closed form of the energy-
   minimising basis, Section 2.2, restricted to a patch neighbourhood).
   Whole patches make Phi^T Psi = I exact.
6. A^(k) = Psi^T A^(k-1) Psi, M^(k) = Psi^T M^(k-1) Psi (Section 2.3 and the
   Lemma on M^(k)), with symbolic (never pruned) patterns, symmetrised.
7. Stop when N^(k) <= n_coarse, k = k_max, or the level does not shrink.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from workloads import CSR


@dataclasses.dataclass
class BuildOpts:
    s_max: int = 8  # seed patch size cap (pass 1); pass-2 joins allowed while size < 2 s_max
    omega_max: int = 256  # row cap of a localisation neighbourhood Omega_j
    loc_radius: int = 1  # 0: Omega_j = P_j, r >= 1: P_j plus r rings of neighbouring patches (r > 1: level 1)
    peel: float = 0.0  # > 0: split off weakly attached rows while 1/lambda_2(patch) > peel * median
    n_coarse: int = 300
    k_max: int = 8
    not_psd_tol: float = 1e-10  # interior energy is "not PSD" if lambda_min < -tol * max|lambda|


@dataclasses.dataclass
class Level:
    """Level k >= 1 of the decomposition."""

    n_fine: int  # N^(k-1)
    n: int  # N^(k)
    patch_of: np.ndarray  # int32 [n_fine]
    patch_ptr: np.ndarray  # int32 [n+1]
    patch_rows: np.ndarray  # int32 [n_fine], rows of each patch ascending
    phi: np.ndarray  # float64 [n_fine], aligned with patch_rows
    uhat: np.ndarray  # float64 [n_fine], normalised Householder vectors aligned with patch_rows
    psi: sp.csr_matrix  # N^(k-1) x N^(k)
    omega_ptr: np.ndarray  # int32 [n+1]
    omega_rows: np.ndarray  # int32, rows of Omega_j ascending
    A: sp.csr_matrix  # A^(k)
    M: sp.csr_matrix  # M^(k)
    eps: float  # eps(P^(k))
    delta: float  # delta(P^(k))
    used_closed: int  # patches whose interior energy was not PSD


@dataclasses.dataclass
class MMD:
    A0: sp.csr_matrix
    levels: list  # Level objects for k = 1..K
    opts: BuildOpts

    @property
    def K(self) -> int:
        return len(self.levels)

    def A(self, k: int) -> sp.csr_matrix:
        return self.A0 if k == 0 else self.levels[k - 1].A

    def M(self, k: int):
        return None if k == 0 else self.levels[k - 1].M

    def N(self, k: int) -> int:
        return self.A0.shape[0] if k == 0 else self.levels[k - 1].n


# --------------------------------------------------------------------------
# 1. partition (integer only)
def partition(rowptr: np.ndarray, col: np.ndarray, n: int, s_max: int):
    """Greedy aggregation of the pattern (diagonal excluded).

    Pass 1: rows in ascending order; a row whose neighbours are all
    unassigned seeds a patch of itself plus its first s_max - 1 neighbours
    (ascending column).  Pass 2: each still unassigned row, ascending, joins
    the neighbouring patch holding most of its neighbours (ties: lowest patch
    id) among patches with fewer than 2 s_max rows; if none qualifies it
    seeds a patch with its unassigned neighbours (ascending, up to s_max - 1).
    Patch ids follow creation order.
    """
    rowptr = np.asarray(rowptr)
    col = np.asarray(col)
    patch_of = np.full(n, -1, dtype=np.int64)
    sizes = []

    def nbrs(i):
        c = col[rowptr[i]:rowptr[i + 1]]
        return c[c != i]

    def seed(i, cand):
        pid = len(sizes)
        patch_of[i] = pid
        cnt = 1
        for j in cand:
            if cnt >= s_max:
                break
            if patch_of[j] < 0:
                patch_of[j] = pid
                cnt += 1
        sizes.append(cnt)

    for i in range(n):
        if patch_of[i] >= 0:
            continue
        nb = nbrs(i)
        if np.all(patch_of[nb] < 0):
            seed(i, nb)
    for i in range(n):
        if patch_of[i] >= 0:
            continue
        nb = nbrs(i)
        counts = {}
        for j in nb:
            p = patch_of[j]
            if p >= 0:
                counts[p] = counts.get(p, 0) + 1
        best, bestc = -1, 0
        for p in sorted(counts):
            if sizes[p] < 2 * s_max and counts[p] > bestc:
                best, bestc = p, counts[p]
        if best >= 0:
            patch_of[i] = best
            sizes[best] += 1
        else:
            seed(i, nb)
    npatch = len(sizes)
    order = np.lexsort((np.arange(n), patch_of))
    patch_rows = order.astype(np.int32)
    patch_ptr = np.zeros(npatch + 1, dtype=np.int32)
    patch_ptr[1:] = np.cumsum(np.bincount(patch_of, minlength=npatch))
    return patch_of.astype(np.int32), patch_ptr, patch_rows


def _inv_lambda2(A: sp.csr_matrix, rowabs: np.ndarray, S: np.ndarray, not_psd_tol: float) -> float:
    """1 / lambda_2 of the patch energy of rows S (interior energy, closed
    energy when that is not PSD), the patch's share of eps(P) (Section 2.2)."""
    AS = A[S][:, S].toarray()
    inside = np.abs(AS).sum(axis=1)
    E = AS - np.diag(rowabs[S] - inside)
    w = np.linalg.eigvalsh(E)
    if w[0] < -not_psd_tol * np.max(np.abs(w)):
        w = np.linalg.eigvalsh(AS)
    return 1.0 / w[1]


def peel(A: sp.csr_matrix, patch_of, patch_ptr, patch_rows, mult: float, not_psd_tol: float):
    """Bound eps(P) by splitting weakly attached rows off their patches.

    eps(P) is a maximum over patches, so one row that hangs on its patch by
    small weights sets it for the whole level.  With cap = mult x the median
    of 1/lambda_2 over patches of two or more rows (lower median), each patch
    in id order loses, while 1/lambda_2 > cap, the row with the smallest
    interior weight sum_{u in S, u != v} |a_vu| (ties: lowest row); every
    removed row becomes a singleton patch, numbered after all existing
    patches in removal order.  Sums run over the CSR row in column order.
    """
    if mult <= 0:
        return patch_of, patch_ptr, patch_rows
    n = A.shape[0]
    rowabs = np.array([sum(abs(float(v)) for v in A.data[A.indptr[r]:A.indptr[r + 1]]) for r in range(n)])
    npatch = len(patch_ptr) - 1
    inv = sorted(_inv_lambda2(A, rowabs, patch_rows[patch_ptr[j]:patch_ptr[j + 1]], not_psd_tol)
                 for j in range(npatch) if patch_ptr[j + 1] - patch_ptr[j] > 1)
    if not inv:
        return patch_of, patch_ptr, patch_rows
    cap = mult * inv[(len(inv) - 1) // 2]
    new_of = np.array(patch_of, dtype=np.int64)
    nxt = npatch
    for j in range(npatch):
        S = [int(r) for r in patch_rows[patch_ptr[j]:patch_ptr[j + 1]]]
        while len(S) > 1 and _inv_lambda2(A, rowabs, np.array(S), not_psd_tol) > cap:
            inS = set(S)
            best, bw = -1, 0.0
            for v in S:  # ascending rows: the first minimum is the lowest row
                t = 0.0
                for k in range(A.indptr[v], A.indptr[v + 1]):
                    c = int(A.indices[k])
                    if c != v and c in inS:
                        t += abs(float(A.data[k]))
                if best < 0 or t < bw:
                    best, bw = v, t
            S.remove(best)
            new_of[best] = nxt
            nxt += 1
    order = np.lexsort((np.arange(n), new_of))
    ptr = np.zeros(nxt + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(np.bincount(new_of, minlength=nxt))
    return new_of.astype(np.int32), ptr, order.astype(np.int32)


# --------------------------------------------------------------------------
# 2-4. local bases
def _sign_fix(v: np.ndarray) -> np.ndarray:
    a = np.abs(v)
    i = int(np.argmax(a))  # first index of the maximum
    return v if v[i] > 0 else -v


def local_bases(A: sp.csr_matrix, patch_ptr, patch_rows, not_psd_tol: float):
    """phi_j, normalised Householder vectors, eps(P), delta(P) (Section 2.2-2.3)."""
    n_fine = A.shape[0]
    npatch = len(patch_ptr) - 1
    phi = np.zeros(n_fine)
    uhat = np.zeros(n_fine)
    absA = abs(A)
    rowabs = np.asarray(absA.sum(axis=1)).ravel()
    eps, delta, used_closed = 0.0, 0.0, 0
    for j in range(npatch):
        S = patch_rows[patch_ptr[j]:patch_ptr[j + 1]]
        AS = A[S][:, S].toarray()
        inside = np.asarray(absA[S][:, S].sum(axis=1)).ravel()
        outside = rowabs[S] - inside  # sum_{j not in S} |a_ij|
        E = AS - np.diag(outside)
        w, V = np.linalg.eigh(E)
        if len(S) > 1 and w[0] < -not_psd_tol * np.max(np.abs(w)):  # a singleton's phi is 1 either way
            used_closed += 1
            E = AS
            w, V = np.linalg.eigh(E)
        p = _sign_fix(V[:, 0])
        phi[patch_ptr[j]:patch_ptr[j + 1]] = p
        if len(S) > 1:
            eps = max(eps, 1.0 / w[1])
        x = np.linalg.solve(AS, p)
        delta = max(delta, 1.0 / float(p @ x))
        u = p.copy()
        u[0] += 1.0 if p[0] >= 0 else -1.0
        uhat[patch_ptr[j]:patch_ptr[j + 1]] = u / np.linalg.norm(u)
    return phi, uhat, eps, delta, used_closed


# --------------------------------------------------------------------------
# 5. localised Psi
def neighbourhoods(A: sp.csr_matrix, patch_of, patch_ptr, patch_rows, omega_max: int, loc_radius: int):
    """Omega_j = P_j plus whole patches in rings around it, integer-only selection.

    Ring 1: the patches holding neighbours of P_j, ranked by the number of
    pattern entries (r, c), r in P_j, c in P_i, c != r (descending; ties:
    lowest patch id).  Ring t >= 2: the patches adjacent to a patch taken in
    ring t - 1 that no earlier ring offered, ascending id.  A patch is added
    while the row count stays <= omega_max (a patch that does not fit is
    skipped and the next one tried).
    """
    npatch = len(patch_ptr) - 1
    rowptr, col = A.indptr, A.indices
    adj = None
    if loc_radius >= 2:
        adj = [set() for _ in range(npatch)]
        for r in range(A.shape[0]):
            pr = int(patch_of[r])
            for c in col[rowptr[r]:rowptr[r + 1]]:
                pc = int(patch_of[c])
                if pc != pr:
                    adj[pr].add(pc)
    optr = [0]
    orows = []
    for j in range(npatch):
        S = patch_rows[patch_ptr[j]:patch_ptr[j + 1]]
        chosen = [j]
        total = len(S)
        if loc_radius >= 1:
            counts = {}
            for r in S:
                for c in col[rowptr[r]:rowptr[r + 1]]:
                    if c == r:
                        continue
                    p = int(patch_of[c])
                    if p != j:
                        counts[p] = counts.get(p, 0) + 1
            ranked = sorted(counts.items(), key=lambda t: (-t[1], t[0]))
            seen = {j} | set(counts)
            ring = []
            for p, _ in ranked:
                sz = int(patch_ptr[p + 1] - patch_ptr[p])
                if total + sz <= omega_max:
                    chosen.append(p)
                    ring.append(p)
                    total += sz
            for _ in range(2, loc_radius + 1):
                cand = sorted({q for p in ring for q in adj[p]} - seen)
                seen.update(cand)
                ring = []
                for p in cand:
                    sz = int(patch_ptr[p + 1] - patch_ptr[p])
                    if total + sz <= omega_max:
                        chosen.append(p)
                        ring.append(p)
                        total += sz
        rows = np.sort(np.concatenate([patch_rows[patch_ptr[p]:patch_ptr[p + 1]] for p in chosen]))
        orows.append(rows)
        optr.append(optr[-1] + len(rows))
    return np.asarray(optr, dtype=np.int32), np.concatenate(orows).astype(np.int32)


def localized_psi(A: sp.csr_matrix, patch_of, patch_ptr, patch_rows, phi, omega_ptr, omega_rows) -> sp.csr_matrix:
    """psi_j from the constrained energy minimisation on Omega_j (KKT, closed form)."""
    n_fine = A.shape[0]
    npatch = len(patch_ptr) - 1
    phi_of_row = np.zeros(n_fine)
    phi_of_row[patch_rows] = phi
    cols, rows, vals = [], [], []
    for j in range(npatch):
        O = omega_rows[omega_ptr[j]:omega_ptr[j + 1]]
        AO = A[O][:, O].toarray()
        pats = patch_of[O]
        plist = np.unique(pats)
        C = np.zeros((len(plist), len(O)))
        for a, p in enumerate(plist):
            m = pats == p
            C[a, m] = phi_of_row[O[m]]
        cf = sla.cho_factor(AO, lower=True)
        Y = sla.cho_solve(cf, C.T)
        S = C @ Y
        e = (plist == j).astype(np.float64)
        psi = Y @ np.linalg.solve(S, e)
        rows.append(O)
        cols.append(np.full(len(O), j))
        vals.append(psi)
    Psi = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_fine, npatch))
    Psi.sort_indices()
    return Psi


# --------------------------------------------------------------------------
# 6. symbolic-pattern Galerkin products
def _pattern(m: sp.spmatrix) -> sp.csr_matrix:
    m = m.tocsr()
    return sp.csr_matrix((np.ones(m.nnz), m.indices, m.indptr), shape=m.shape)


def values_on_pattern(pat: sp.csr_matrix, num: sp.csr_matrix) -> np.ndarray:
    """Values of ``num`` at the positions of ``pat`` (0 where num has none)."""
    pat = pat.tocsr()
    pat.sort_indices()
    num = num.tocsr()
    num.sort_indices()
    n = pat.shape[1]
    prow = np.repeat(np.arange(pat.shape[0], dtype=np.int64), np.diff(pat.indptr))
    nrow = np.repeat(np.arange(num.shape[0], dtype=np.int64), np.diff(num.indptr))
    pkey = prow * n + pat.indices
    nkey = nrow * n + num.indices
    pos = np.searchsorted(nkey, pkey)
    pos = np.minimum(pos, max(len(nkey) - 1, 0))
    out = np.zeros(len(pkey))
    if len(nkey):
        hit = nkey[pos] == pkey
        out[hit] = num.data[pos[hit]]
    return out


def galerkin(Psi: sp.csr_matrix, B: sp.csr_matrix | None) -> sp.csr_matrix:
    """Psi^T B Psi (B = None means identity) on its symbolic pattern, symmetrised."""
    if B is None:
        num = (Psi.T @ Psi).tocsr()
        pat = (_pattern(Psi).T @ _pattern(Psi)).tocsr()
    else:
        num = (Psi.T @ (B @ Psi)).tocsr()
        pat = (_pattern(Psi).T @ (_pattern(B) @ _pattern(Psi))).tocsr()
    pat.sort_indices()
    v = values_on_pattern(pat, num)
    vt = values_on_pattern(pat, num.T.tocsr())
    out = sp.csr_matrix((0.5 * (v + vt), pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)
    return out


# --------------------------------------------------------------------------
def build_level(A: sp.csr_matrix, Mprev, opts: BuildOpts, k: int = 1) -> Level:
    """Level k from level k - 1.  Wider supports (loc_radius > 1) apply to
    level 1 only; deeper levels use at most one ring (their Galerkin matrices
    are dense enough that two rings reach omega_max)."""
    A = A.tocsr()
    A.sort_indices()
    n_fine = A.shape[0]
    patch_of, patch_ptr, patch_rows = partition(A.indptr, A.indices, n_fine, opts.s_max)
    patch_of, patch_ptr, patch_rows = peel(A, patch_of, patch_ptr, patch_rows, opts.peel, opts.not_psd_tol)
    phi, uhat, eps, delta, used_closed = local_bases(A, patch_ptr, patch_rows, opts.not_psd_tol)
    radius = opts.loc_radius if k == 1 else min(opts.loc_radius, 1)
    optr, orows = neighbourhoods(A, patch_of, patch_ptr, patch_rows, opts.omega_max, radius)
    Psi = localized_psi(A, patch_of, patch_ptr, patch_rows, phi, optr, orows)
    Ak = galerkin(Psi, A)
    Mk = galerkin(Psi, Mprev)
    return Level(n_fine, len(patch_ptr) - 1, patch_of, patch_ptr, patch_rows, phi, uhat, Psi, optr, orows,
                 Ak, Mk, eps, delta, used_closed)


def build(A: CSR | sp.csr_matrix, opts: BuildOpts | None = None) -> MMD:
    """Full decomposition: levels k = 1..K until the stopping rule holds."""
    opts = opts or BuildOpts()
    A0 = A.to_scipy() if isinstance(A, CSR) else A.tocsr()
    A0.sort_indices()
    levels = []
    cur, Mcur = A0, None
    while cur.shape[0] > opts.n_coarse and len(levels) < opts.k_max:
        lev = build_level(cur, Mcur, opts, len(levels) + 1)
        if lev.n >= cur.shape[0]:
            break
        levels.append(lev)
        cur, Mcur = lev.A, lev.M
    return MMD(A0, levels, opts)


# --------------------------------------------------------------------------
# Householder complement U^(k) (Section 2.3 and 5): coordinates of patch j are
# positions 1..|P_j|-1 of H_j, i.e. complement index patch_ptr[j] - j + (t - 1).
def U_apply(lev: Level, g: np.ndarray) -> np.ndarray:
    """y = U g, g of length N^(k-1) - N^(k) (columns may be a 2D block)."""
    g = np.asarray(g, dtype=np.float64)
    shape = (lev.n_fine,) + g.shape[1:]
    y = np.zeros(shape)
    for j in range(lev.n):
        a, b = lev.patch_ptr[j], lev.patch_ptr[j + 1]
        rows = lev.patch_rows[a:b]
        u = lev.uhat[a:b]
        t = np.zeros((b - a,) + g.shape[1:])
        t[1:] = g[a - j:b - j - 1]
        t = t - 2.0 * np.multiply.outer(u, u @ t) if t.ndim > 1 else t - 2.0 * u * (u @ t)
        y[rows] = t
    return y


def Ut_apply(lev: Level, x: np.ndarray) -> np.ndarray:
    """g = U^T x."""
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros((lev.n_fine - lev.n,) + x.shape[1:])
    for j in range(lev.n):
        a, b = lev.patch_ptr[j], lev.patch_ptr[j + 1]
        rows = lev.patch_rows[a:b]
        u = lev.uhat[a:b]
        t = x[rows]
        t = t - 2.0 * np.multiply.outer(u, u @ t) if t.ndim > 1 else t - 2.0 * u * (u @ t)
        g[a - j:b - j - 1] = t[1:]
    return g


def Phi_matrix(lev: Level) -> sp.csr_matrix:
    """Phi^(k) as an N^(k-1) x N^(k) sparse matrix (column j = phi_j on P_j)."""
    cols = np.repeat(np.arange(lev.n), np.diff(lev.patch_ptr))
    return sp.csr_matrix((lev.phi, (lev.patch_rows, cols)), shape=(lev.n_fine, lev.n))
