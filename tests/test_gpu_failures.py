"""Failure paths of the eigensolver on the GPU, made without a GPU fault.

* A device wait that runs out: the grid barriers of the cooperative kernels
  give up after opts.timeout_s and set a status word; with a limit far below
  the time the other blocks take to arrive the first barrier runs out, the
  kernel returns normally and the call reports MMD_ETIMEOUT.  The context
  stays usable: the next call on the same handle succeeds.
* Iteration caps (max_cg_iter, max_restarts, max_refine_iter = 1): the call
  returns MMD_ENOCONV with the partial pairs and counts the capped loops.
* Options and batched arguments the algorithms cannot use: MMD_EINVAL before
  any work.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _pkg():
    import paper_1804_03415_gb300 as pkg

    return pkg


def test_device_wait_timeout_then_recovers():
    pkg = _pkg()
    A = W.torus_knn(3000, seed=W.BASE_SEED + 70)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=80)
    with pytest.raises(pkg.MMDError) as ei:
        h.eig_leftmost(10, 1e-8, timeout_s=1e-9)
    assert ei.value.code == pkg._lib.MMD_ETIMEOUT
    lam, V, st = h.eig_leftmost(10, 1e-8)
    ev = np.linalg.eigvalsh(A.dense())[:10]
    assert np.abs(lam - ev).max() <= 1e-9 * np.abs(ev).max() + 1e-12 * np.abs(A.val).max()
    assert st["max_rel_residual"] <= 10 * 1e-8
    h.close()


def test_iteration_caps_return_partial_results():
    pkg = _pkg()
    A = W.fd2d(24, seed=W.BASE_SEED + 71)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=50)
    with pytest.raises(pkg.MMDError) as ei:
        h.eig_leftmost(12, 1e-10, max_cg_iter=1, max_restarts=1, max_refine_iter=1)
    assert ei.value.code == pkg._lib.MMD_ENOCONV
    lam, V, st = h.eig_leftmost(12, 1e-10, allow_noconv=True, max_cg_iter=1, max_restarts=1, max_refine_iter=1)
    assert st["not_converged"] > 0 and st["nc_solve"] > 0
    assert st["not_converged"] == st["nc_solve"] + st["nc_restart"] + st["nc_refine"]
    assert st["n_converged"] < 12
    assert lam.shape == (12,) and np.all(np.isfinite(lam))
    # the handle is still usable and exact afterwards
    lam, V, st = h.eig_leftmost(12, 1e-10)
    ev = np.linalg.eigvalsh(A.dense())[:12]
    assert np.abs(lam - ev).max() <= 1e-9 * np.abs(ev).max()
    h.close()


@pytest.mark.parametrize("bad", [{"alpha": 0.0}, {"beta": -1.0}, {"c_r": 0}, {"max_cg_iter": 0},
                                 {"timeout_s": 0.0}, {"precision": 7}, {"d": -2}, {"poly_op": 33},
                                 {"poly_refine": -1}, {"poly_ratio": 1.0}, {"mg_op": 9}])
def test_invalid_options_refused_by_every_entry_point(bad):
    pkg = _pkg()
    A = W.fd2d(10, seed=W.BASE_SEED + 72)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=20)
    with pytest.raises(pkg.MMDError) as ei:
        h.eig_leftmost(3, 1e-8, **bad)
    assert ei.value.code == pkg._lib.MMD_EINVAL
    B = W.fd2d(9, seed=W.BASE_SEED + 73)
    h2 = pkg.MMD(B.rowptr, B.col, B.val, n_coarse=20)
    with pytest.raises(pkg.MMDError) as ei:
        pkg.eig_leftmost_batched([h, h2], [3, 3], 1e-8, **bad)
    assert ei.value.code == pkg._lib.MMD_EINVAL
    h.eig_leftmost(3, 1e-10)
    with pytest.raises(pkg.MMDError) as ei:
        h.eig_grad(np.ones(3), None, **bad)
    assert ei.value.code == pkg._lib.MMD_EINVAL
    h.close()
    h2.close()


def test_batched_refuses_shared_handles():
    pkg = _pkg()
    A = W.fd2d(10, seed=W.BASE_SEED + 74)
    h = pkg.MMD(A.rowptr, A.col, A.val, n_coarse=20)
    with pytest.raises(pkg.MMDError) as ei:
        pkg.eig_leftmost_batched([h, h], [3, 3], 1e-8)
    assert ei.value.code == pkg._lib.MMD_EINVAL
    assert "share one handle" in str(ei.value)
    h.close()
