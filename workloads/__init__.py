"""Seeded synthetic SPD matrices shared by the oracle, the tests and the bench.

This module builds inputs only.  It holds none of the eigensolver's arithmetic
(no decomposition, no solver, no eigen-step): every function here returns a
symmetric sparse matrix in full CSR storage (sorted column indices, diagonal
stored) so that both the CPU oracle and the CUDA library read identical bytes.

Workloads (sizes follow the paper's kind of inputs; none are the paper's data):

* ``fd2d``       -- 2D 5-point finite-difference operator -div(a grad u) with
  Dirichlet boundary, cell-centred unknowns, h = 1, interior face coefficient
  = harmonic mean of the two cells, boundary face coefficient = the cell's a.
  With a == 1 it is the textbook (4, -1) stencil.
* ``fd3d``       -- the same in 3D (7-point), optional high-contrast inclusion
  boxes (axis-aligned, sides uniform in {4..16}, until >= 10% of cells).
* ``torus_knn``  -- symmetric kNN graph Laplacian of points sampled
  area-uniformly on a torus (R, r) with Gaussian jitter, weights
  exp(-d^2/sigma^2), sigma = mean directed kNN distance, plus shift * I.
  Stand-in for the paper's kNN point-cloud graphs (Section 7.1).
* ``rgg``        -- random geometric graph Laplacian in the unit square,
  radius sqrt(deg / (pi n)), optional U(lo, hi) weights, optional restriction
  to the largest connected component, plus shift * I.
* ``swissroll``  -- the paper's SwissRoll point cloud (Section 7.1) as a kNN
  graph with weights exp(-r^2 / sigma).

Random numbers come from ``numpy.random.default_rng(seed)``; the canonical
seed of workload index c is ``1804034150 + c``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 1804034150


@dataclasses.dataclass
class CSR:
    """Symmetric matrix in full CSR storage (int32 indices, float64 values)."""

    n: int
    rowptr: np.ndarray  # int32, n + 1
    col: np.ndarray  # int32, nnz, sorted within each row
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Sum duplicates, sort columns, return CSR with int32 indices."""
    import scipy.sparse as sp

    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    if m.nnz >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64))


def laplacian_from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray, shift: float) -> CSR:
    """Graph Laplacian D - W (+ shift I) of undirected edges (i, j, w), i != j, each once."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    w = np.asarray(w, np.float64)
    deg = np.bincount(i, weights=w, minlength=n) + np.bincount(j, weights=w, minlength=n)
    diag = np.arange(n, dtype=np.int64)
    rows = np.concatenate([i, j, diag])
    cols = np.concatenate([j, i, diag])
    vals = np.concatenate([-w, -w, deg + shift])
    return _from_coo(n, rows, cols, vals)


# ---------------------------------------------------------------- FD operators
def _fd_from_cells(a: np.ndarray) -> CSR:
    """Cell-centred FD operator for coefficient field ``a`` of any dimension."""
    shape = a.shape
    n = a.size
    idx = np.arange(n, dtype=np.int64).reshape(shape)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for ax in range(a.ndim):
        lo = [slice(None)] * a.ndim
        hi = [slice(None)] * a.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        a0, a1 = a[tuple(lo)], a[tuple(hi)]
        face = 2.0 * a0 * a1 / (a0 + a1)
        i0, i1 = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        f = face.ravel()
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-f, -f]
        np.add.at(diag, i0, f)
        np.add.at(diag, i1, f)
        # Dirichlet boundary faces on both ends of this axis
        first = [slice(None)] * a.ndim
        last = [slice(None)] * a.ndim
        first[ax] = 0
        last[ax] = -1
        np.add.at(diag, idx[tuple(first)].ravel(), a[tuple(first)].ravel())
        np.add.at(diag, idx[tuple(last)].ravel(), a[tuple(last)].ravel())
    d = np.arange(n, dtype=np.int64)
    rows.append(d)
    cols.append(d)
    vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def fd2d(m: int, seed: int = BASE_SEED + 0, log10_range=(-2.0, 2.0), const: bool = False) -> CSR:
    """m x m cells, a = 10^U(lo, hi) i.i.d. per cell (or a == 1 when ``const``)."""
    if const:
        a = np.ones((m, m))
    else:
        rng = np.random.default_rng(seed)
        a = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=(m, m))
    return _fd_from_cells(a)


def fd3d(m: int, seed: int = BASE_SEED + 2, log10_range=(-3.0, 3.0), inclusions: bool = True,
         const: bool = False, inclusion_value: float = 1e4, cover: float = 0.10) -> CSR:
    """m^3 cells, a = 10^U(lo, hi), plus inclusion boxes set to ``inclusion_value``."""
    if const:
        return _fd_from_cells(np.ones((m, m, m)))
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=(m, m, m))
    if inclusions:
        mask = np.zeros((m, m, m), bool)
        target = cover * m**3
        while mask.sum() < target:
            side = rng.integers(4, 17, size=3)
            side = np.minimum(side, m)
            org = [int(rng.integers(0, m - s + 1)) for s in side]
            mask[org[0]:org[0] + side[0], org[1]:org[1] + side[1], org[2]:org[2] + side[2]] = True
        a[mask] = inclusion_value
    return _fd_from_cells(a)


# -------------------------------------------------------------------- graphs
def _knn_union_edges(pts: np.ndarray, k: int):
    from scipy.spatial import cKDTree

    tree = cKDTree(pts)
    d, nb = tree.query(pts, k=k + 1)
    d, nb = d[:, 1:], nb[:, 1:]
    n = pts.shape[0]
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    dst = nb.ravel().astype(np.int64)
    dist = d.ravel()
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    key = lo * n + hi
    key, first = np.unique(key, return_index=True)
    return lo[first], hi[first], dist[first], d


def torus_knn(npts: int, k: int = 10, seed: int = BASE_SEED + 1, R: float = 1.0, r: float = 0.3,
              jitter: float = 1e-3, shift: float = 1e-6) -> CSR:
    """kNN graph Laplacian of ``npts`` area-uniform torus points (union symmetrisation)."""
    rng = np.random.default_rng(seed)
    th = np.empty(0)
    while th.size < npts:
        t = rng.uniform(0.0, 2 * math.pi, size=2 * npts)
        acc = rng.uniform(0.0, 1.0, size=2 * npts) < (R + r * np.cos(t)) / (R + r)
        th = np.concatenate([th, t[acc]])
    th = th[:npts]
    ph = rng.uniform(0.0, 2 * math.pi, size=npts)
    pts = np.stack([(R + r * np.cos(th)) * np.cos(ph), (R + r * np.cos(th)) * np.sin(ph), r * np.sin(th)], 1)
    pts += rng.normal(0.0, jitter, size=pts.shape)
    i, j, dist, dall = _knn_union_edges(pts, k)
    sigma = float(dall.mean())
    w = np.exp(-(dist**2) / sigma**2)
    return laplacian_from_edges(npts, i, j, w, shift)


def rgg(n: int, deg: float = 8.0, seed: int = BASE_SEED + 3, weights=None, lcc: bool = False,
        shift: float = 1e-6) -> CSR:
    """Random geometric graph Laplacian in [0,1]^2, radius sqrt(deg / (pi n)).

    ``weights``: None for unit weights, or (lo, hi) for U(lo, hi) edge weights.
    ``lcc``: keep the largest connected component, relabelled by ascending index.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    rad = math.sqrt(deg / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(rad, output_type="ndarray").astype(np.int64)
    pairs.sort(axis=1)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    pairs = pairs[order]
    if weights is None:
        w = np.ones(len(pairs))
    else:
        w = rng.uniform(weights[0], weights[1], size=len(pairs))
    if lcc:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import connected_components

        adj = sp.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
        _, lab = connected_components(adj, directed=False)
        big = np.argmax(np.bincount(lab))
        keep = lab == big
        newid = -np.ones(n, np.int64)
        newid[keep] = np.arange(keep.sum())
        sel = keep[pairs[:, 0]] & keep[pairs[:, 1]]
        pairs, w = pairs[sel], w[sel]
        pairs = newid[pairs]
        n = int(keep.sum())
    return laplacian_from_edges(n, pairs[:, 0], pairs[:, 1], w, shift)


def rgg_batch(count: int = 64, seed: int = BASE_SEED + 3, lo: int = 2000, hi: int = 50000, deg: float = 8.0):
    """``count`` RGG Laplacians (+1e-6 I), sizes floor(exp(U(ln lo, ln hi))), unit weights."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(int)
    return [rgg(int(s), deg=deg, seed=seed + 1000 * (b + 1)) for b, s in enumerate(sizes)]


def swissroll(n: int = 20000, k: int = 10, seed: int = BASE_SEED + 5, sigma: float = 0.1,
              noise_var: float = 0.05, shift: float = 1e-6) -> CSR:
    """SwissRoll kNN graph: t ~ U[1.5pi, 4.5pi], y ~ U[0, 20], noise N(0, noise_var I3)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(1.5 * math.pi, 4.5 * math.pi, size=n)
    y = rng.uniform(0.0, 20.0, size=n)
    pts = np.stack([t * np.cos(t), y, t * np.sin(t)], 1) + rng.normal(0.0, math.sqrt(noise_var), size=(n, 3))
    i, j, dist, _ = _knn_union_edges(pts, k)
    w = np.exp(-(dist**2) / sigma)
    return laplacian_from_edges(n, i, j, w, shift)


def path_graph(n: int, shift: float = 0.0) -> CSR:
    """Path graph Laplacian on n nodes (unit weights)."""
    i = np.arange(n - 1)
    return laplacian_from_edges(n, i, i + 1, np.ones(n - 1), shift)


def random_spd_mmatrix(n: int, deg: float, seed: int, shift: float = 1e-2) -> CSR:
    """Small random weighted graph Laplacian + shift I (an SPD M-matrix) for fuzz tests."""
    rng = np.random.default_rng(seed)
    m = int(n * deg / 2)
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    i, j = np.minimum(i[keep], j[keep]), np.maximum(i[keep], j[keep])
    key = np.unique(i.astype(np.int64) * n + j)
    i, j = key // n, key % n
    w = rng.uniform(0.5, 2.0, size=len(i))
    return laplacian_from_edges(n, i, j, w, shift)


# Named workloads (index c uses seed BASE_SEED + c).
def workload(name: str) -> CSR:
    if name == "fd2d_64":
        return fd2d(64, seed=BASE_SEED + 0)
    if name == "torus_knn_200k":
        return torus_knn(200_000, seed=BASE_SEED + 1)
    if name == "fd3d_128":
        return fd3d(128, seed=BASE_SEED + 2)
    if name == "rgg_50k":
        return rgg(50_000, deg=10.0, seed=BASE_SEED + 4, weights=(0.5, 2.0), lcc=True)
    if name == "swissroll_20k":
        return swissroll(20_000)
    raise KeyError(name)
