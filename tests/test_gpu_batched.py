"""eig_leftmost_batched: independent problems solved concurrently on several
streams give the same eigenpairs as the oracle's dense eigensolver (the
batched path shares no state between problems, so each result is checked on
its own)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_batched_matches_dense():
    import paper_1804_03415_gb300 as pkg

    mats = [W.fd2d(14, seed=W.BASE_SEED + 41), W.fd2d(16, const=True),
            W.rgg(700, deg=10.0, seed=W.BASE_SEED + 42, weights=(0.5, 2.0), lcc=True),
            W.fd2d(12, seed=W.BASE_SEED + 43), W.rgg(500, deg=9.0, seed=W.BASE_SEED + 44, lcc=True)]
    Ns = [6, 5, 8, 4, 7]
    tol = 1e-10
    hs = [pkg.MMD(A.rowptr, A.col, A.val, n_coarse=40) for A in mats]
    out = pkg.eig_leftmost_batched(hs, Ns, tol, streams=3)
    for A, N, (lam, V, st) in zip(mats, Ns, out):
        lo = np.linalg.eigvalsh(A.dense())
        nA = np.abs(A.dense()).sum(1).max()
        assert st["n_converged"] >= N
        assert np.abs(lam - lo[:N]).max() <= 1e-8 * nA
        R = A.to_scipy() @ V - V * lam
        assert np.linalg.norm(R, axis=0).max() <= 10 * tol * nA
        assert np.abs(V.T @ V - np.eye(N)).max() <= 1e-9
    for h in hs:
        h.close()


def test_batched_rejects_bad_problem():
    import paper_1804_03415_gb300 as pkg

    A = W.fd2d(10, seed=W.BASE_SEED + 45)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=20)
    with pytest.raises(pkg.MMDError):
        pkg.eig_leftmost_batched([h, h], [3, A.n + 1], 1e-8)
    h.close()
