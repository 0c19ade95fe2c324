"""Write tests/golden/torus_knn_200k_eigs.json: the 520 smallest eigenvalues
of the torus kNN 200k workload (the benchmark's matrix) from the oracle's
independent shift-invert Lanczos check (oracle/reference.py), with the
sha256 of the input CSR and checks that also hold across machines whose
libm rounds exp() differently in the last bit (the sha256 of the integer
pattern, and the sum and sum of squares of the values).

    python tests/golden/make_torus_knn_200k_eigs.py      # ~10-20 min on 8 cores
"""
import datetime
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import scipy  # noqa: E402

import workloads as W  # noqa: E402
from oracle import reference as OR  # noqa: E402

NEV = 520


def main():
    A = W.torus_knn(200_000, k=10, seed=W.BASE_SEED + 1)
    h = hashlib.sha256()
    for arr in (A.rowptr, A.col, A.val):
        h.update(np.ascontiguousarray(arr).tobytes())
    hp = hashlib.sha256()
    for arr in (A.rowptr, A.col):
        hp.update(np.ascontiguousarray(arr).tobytes())
    t0 = time.time()
    lam, V = OR.leftmost_shift_invert(A.to_scipy(), NEV)
    el = time.time() - t0
    S = A.to_scipy()
    res = np.linalg.norm(S @ V - V * lam, axis=0)
    ninf = float(np.abs(S).sum(axis=1).max())
    out = {
        "_about": "smallest eigenvalues of torus_knn(200000, k=10, seed=1804034151) by shift-invert Lanczos "
                  "(oracle/reference.py); written by tests/golden/make_torus_knn_200k_eigs.py",
        "method": "scipy eigsh shift-invert about 0 (ARPACK) with a SuperLU factorisation, tol 1e-13",
        "input_sha256": h.hexdigest(), "pattern_sha256": hp.hexdigest(),
        "val_sum": float(np.sum(A.val)), "val_sq_sum": float(np.sum(A.val ** 2)),
        "n": int(A.n), "nnz": int(A.nnz), "norm_A_inf": ninf,
        "max_residual_over_normA": float(res.max() / ninf),
        "eigenvalues": [float(x) for x in lam],
        "when": datetime.date.today().isoformat(), "seconds": round(el, 1), "scipy": scipy.__version__,
        "machine": platform.machine(), "cores": os.cpu_count(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "torus_knn_200k_eigs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, el, res.max() / ninf)


if __name__ == "__main__":
    main()
