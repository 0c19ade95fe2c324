"""eig_leftmost_batched: independent problems solved concurrently on several
streams give, problem by problem, the oracle's eigenpairs (the batched path
shares no state between problems, so each result is checked on its own) at
the tolerances of the single-problem parity test: relative eigenvalue error
<= max(1e-9, 10 u ||A|| / lambda_i) (the second term bounds what FP64 can
resolve for the 1e-6-shifted zero modes of a graph Laplacian) and cluster
subspaces with every principal-angle cosine >= 1 - 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import eig as OE
from oracle import mmd as OM

pytestmark = pytest.mark.gpu

U64 = np.finfo(np.float64).eps


def _clusters(lam, rel=1e-6):
    out, cur = [], [0]
    for i in range(1, len(lam)):
        if abs(lam[i] - lam[i - 1]) <= rel * max(abs(lam[i]), abs(lam[i - 1])):
            cur.append(i)
        else:
            out.append(cur)
            cur = [i]
    out.append(cur)
    return out


def test_batched_matches_oracle():
    import paper_1804_03415_gb300 as pkg

    mats = [W.fd2d(14, seed=W.BASE_SEED + 41), W.fd2d(16, const=True),
            W.rgg(700, deg=10.0, seed=W.BASE_SEED + 42, weights=(0.5, 2.0), lcc=True),
            W.fd2d(12, seed=W.BASE_SEED + 43), W.rgg(500, deg=9.0, seed=W.BASE_SEED + 44, lcc=True),
            W.rgg(900, deg=8.0, seed=W.BASE_SEED + 46)]
    Ns = [6, 5, 8, 4, 7, 9]
    tol = 1e-10
    nc = 40
    hs = [pkg.MMD(A.rowptr, A.col, A.val, n_coarse=nc) for A in mats]
    out = pkg.eig_leftmost_batched(hs, Ns, tol, streams=3)
    for b, (A, N, (lam, V, st)) in enumerate(zip(mats, Ns, out)):
        ref = OE.eig_leftmost(OM.build(A, OM.BuildOpts(n_coarse=nc)), N, tol)
        nA = np.abs(A.dense()).sum(1).max()
        rtol = np.maximum(1e-9, 10 * U64 * nA / np.abs(ref.lam))
        rel = np.abs(lam - ref.lam) / np.abs(ref.lam)
        assert np.all(rel <= rtol), (b, rel, rtol)
        lam_all = np.linalg.eigvalsh(A.dense())
        for cl in _clusters(ref.lam):
            if cl[-1] == N - 1 and abs(lam_all[N] - ref.lam[-1]) <= 1e-6 * abs(lam_all[N]):
                continue  # a cluster cut by N: only the whole cluster's span is unique
            s = np.linalg.svd(V[:, cl].T @ ref.V[:, cl], compute_uv=False)
            assert s.min() >= 1 - 1e-12, (b, cl, s.min())
        assert st["n_converged"] >= N
        R = A.to_scipy() @ V - V * lam
        assert np.linalg.norm(R, axis=0).max() <= 10 * tol * nA
        assert np.abs(V.T @ V - np.eye(N)).max() <= 1e-9
    for h in hs:
        h.close()


def test_batched_rejects_bad_problem():
    import paper_1804_03415_gb300 as pkg

    A = W.fd2d(10, seed=W.BASE_SEED + 45)
    B = W.fd2d(9, seed=W.BASE_SEED + 47)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=20)
    h2 = pkg.MMD(B.rowptr, B.col, B.val, n_coarse=20)
    with pytest.raises(pkg.MMDError):
        pkg.eig_leftmost_batched([h, h2], [3, B.n + 1], 1e-8)
    h.close()
    h2.close()
