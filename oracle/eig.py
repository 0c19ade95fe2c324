"""Oracle: the hierarchical eigensolver (Algorithms 2-6), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper works with mu = 1/lambda (eigenvalues of A^{-1}, descending) and,
on level k, with coefficient vectors V-hat in the basis Psi^(k), which are
M^(k)-orthonormal (Section 4, end).  The level operator is
(A^(k))^{-1} M^(k) (Lemma 3.2), applied through Operator OP.

Readings of points the paper leaves open (each is also listed in the design
notes of the repository):

* Level-0 completion: the paper stops at level 1 (accuracy eps_1).  To reach
  a residual target the loop of Algorithm 6 continues to k = 0 with
  A^(0) = A, M^(0) = I, Psi^(1) transfer, refinement threshold
  mu_re^(0) = alpha eps_1 and no extension threshold (extend to m_tar).
* Units.  The paper normalises mu_1 = 1 (Section 7.1).  Here absolute
  thresholds (eps_k, mu_re, mu_ex, Lanczos residuals) stay in mu units and
  relative quantities (PCG tolerance, subspace-change test) use eps_k / mu_1
  with mu_1 the largest eigenvalue found on the coarsest level.  On level 0
  the tests are relative to the target: PCG 0.1 tol, Ritz residual
  <= tol * theta_i, subspace change < tol.
* Lanczos breakdown (Algorithm 3): ||f||_M < 1e-10 ||w||_M draws a seeded
  random vector, M-orthogonalised against [V_ini, V]; the T coupling is 0.
* Re-orthogonalisation: two classical Gram-Schmidt passes in the M inner
  product against [V_ini, V]; only alpha_j = h_j enters T.
* Implicit restart (Algorithm 2): exact shifts = the p smallest Ritz values
  of T_{k+p} computed after the p-step extension; f update uses the
  pre-truncation basis.
* "c . d steps of shifts" (Algorithm 4): p = max(c_r d, k) with c_r = 1, k the
  current dimension (the factorisation doubles before the shifts, as in ARPACK;
  with the paper's d = N/10 a single shift per restart stalls for small N).
* Refinement window (Algorithm 5, renew m_h): besides mu_mh >= mu_re, keep
  mu_mh >= mu_ml alpha / (1 + beta), the ratio of the efficiency condition (ii)
  of Section 6, so the first m_h columns converge even when the coarser level
  stopped on the pair count instead of mu_ex.
* Lanczos residual: ||f||_M |e_k^T y_i| maximised, inside the search loop of
  Algorithm 4, over the Ritz pairs above the search buffer (all but the d
  smallest Ritz values of T, the buffer that mu-hat is read from, which the
  next d-step extension keeps refining) and, in the loop after it (whose
  Schur vectors are the output), over all Ritz pairs of T.
* M-QR in Algorithm 5: column-scaled CholQR2 in the M inner product.
* S = W^T F is symmetrised before its eigen-decomposition (descending).
* Refinement stop: ||Q_mh - Q'_mh (Q'_mh^T M Q_mh)||_F < eps / sqrt(1 + eps_h delta_h)
  (the stricter of the two forms in Section 5).
* Coarsest level: keep the pairs with mu >= beta eps_K, at most m_tar.
* d = max(1, min(floor(N^(k)/10), floor(m_tar/10))) (Section 6) on levels with an
  extension threshold; where there is none (level 0, the last level computed)
  the searching step has nothing to search and d = m_tar - dim V_ini.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import mmd as _mmd
from . import rng as _rng
from .solvers import Counters, bsolve, fpcg, op


@dataclasses.dataclass
class EigOpts:
    alpha: float = 3.0
    beta: float = 1.0
    c_r: int = 1
    d: int = 0  # 0: automatic (Section 6)
    max_cg_iter: int = 20000
    max_restarts: int = 400
    max_refine_iter: int = 100
    seed: int = 20180409
    breakdown: float = 1e-10
    method: str = "hierarchical"  # or "irlm_cg": Section 8's baseline (no decomposition)
    stop_level: int = 0  # last level computed; s >= 1 returns Psi^(1)...Psi^(s) V^(s) (accuracy eps_s)


@dataclasses.dataclass
class LevelStats:
    k: int
    n: int
    m_refined: int = 0
    m_extended: int = 0
    refine_iters: int = 0
    restarts: int = 0
    lanczos_steps: int = 0


# --------------------------------------------------------------------------
def _mdot(M, X, Y):
    return X.T @ (Y if M is None else M @ Y)


def _apply_M(M, x):
    return x if M is None else M @ x


class Lanczos:
    """M-Lanczos factorisation (Algorithm 3) with locked columns V_ini."""

    def __init__(self, M, Vini, f, seed, stream0, breakdown):
        self.M = M
        self.Vini = Vini
        self.V = np.zeros((f.shape[0], 0))
        self.alpha = []
        self.beta = []  # beta[i] couples Lanczos vectors i and i+1
        self.f = f
        self.wnorm = None
        self.seed = seed
        self.stream = stream0
        self.breakdown = breakdown
        self.steps = 0

    @property
    def j(self):
        return self.V.shape[1]

    def basis(self):
        return np.hstack([self.Vini, self.V])

    def orth(self, f):
        B = self.basis()
        for _ in range(2):
            f = f - B @ _mdot(self.M, B, f)
        return f

    def fnorm(self):
        return float(np.sqrt(self.f @ _apply_M(self.M, self.f)))

    def step(self, opfun):
        bta = self.fnorm()
        coupling = bta
        if self.wnorm is not None and bta < self.breakdown * self.wnorm:
            r = _rng.uniform_pm1(self.seed, self.stream, self.f.shape[0])
            self.stream += 1
            self.f = self.orth(r)
            bta = self.fnorm()
            coupling = 0.0
        if self.j > 0:
            self.beta.append(coupling)
        v = self.f / bta
        self.V = np.hstack([self.V, v[:, None]])
        w = opfun(v)
        self.wnorm = float(np.sqrt(w @ _apply_M(self.M, w)))
        B = self.basis()
        h = _mdot(self.M, B, w)
        f = w - B @ h
        h2 = _mdot(self.M, B, f)
        f = f - B @ h2
        h = h + h2
        self.alpha.append(float(h[-1]))
        self.f = f
        self.steps += 1

    def T(self):
        j = self.j
        T = np.diag(np.asarray(self.alpha[:j]))
        if j > 1:
            b = np.asarray(self.beta[:j - 1])
            T += np.diag(b, 1) + np.diag(b, -1)
        return T

    def ritz(self):
        th, Y = np.linalg.eigh(self.T())
        res = self.fnorm() * np.abs(Y[-1, :])
        return th, Y, res

    def restart(self, k, p):
        """Algorithm 2 on a factorisation of k + p columns: p exact shifts, keep k."""
        T = self.T()
        assert T.shape[0] == k + p
        th = np.linalg.eigvalsh(T)
        shifts = th[:p]
        Q = np.eye(k + p)
        I = np.eye(k + p)
        for s in shifts:
            Qj, Rj = np.linalg.qr(T - s * I)
            T = Rj @ Qj + s * I
            Q = Q @ Qj
        Vold = self.V
        self.V = Vold @ Q[:, :k]
        self.f = Vold @ Q[:, k] * T[k, k - 1] + self.f * Q[k + p - 1, k - 1]
        Ts = 0.5 * (T + T.T)
        self.alpha = list(np.diag(Ts)[:k])
        self.beta = list(np.diag(Ts, -1)[:k - 1])
        self.wnorm = None


# --------------------------------------------------------------------------
def extend(A, M, Vini, Dini, pcg_tol, res_ok, mu_ex, d, m_tar, opts: EigOpts, ctr: Counters,
           st: LevelStats, stream0: int):
    """Algorithm 4 (Eigenpair Extension).  res_ok(theta, res) -> bool."""
    m0 = Vini.shape[1]
    if m0 >= m_tar:
        return Vini, Dini
    n = A.shape[0]
    if n - m0 <= 0:
        return Vini, Dini
    if mu_ex is None and opts.d == 0:
        # no extension threshold (level 0, or the last level computed): the
        # searching step only serves the test of mu-hat against mu_ex (Section
        # 6), so one extension goes straight to the target
        d = max(1, m_tar - m0)
    r = _rng.uniform_pm1(opts.seed, stream0, n)
    lz = Lanczos(M, Vini, r, opts.seed, stream0 + 1, opts.breakdown)
    lz.f = lz.orth(r)
    opfun = lambda x: op(A, M, x, pcg_tol, opts.max_cg_iter, ctr)
    room = n - m0  # Krylov space dimension available
    p = max(1, opts.c_r * d)

    def converge(pp, skip):
        # th ascending: the `skip` smallest Ritz values form the search buffer
        for _ in range(opts.max_restarts):
            th, _, res = lz.ritz()
            if res_ok(th[skip:], res[skip:]):
                return
            pp_eff = min(max(pp, lz.j), room - lz.j)
            if pp_eff <= 0:
                return
            k = lz.j
            for _ in range(pp_eff):
                lz.step(opfun)
            lz.restart(k, pp_eff)
            st.restarts += 1
        ctr.not_converged += 1

    while True:
        steps = min(d, room - lz.j)
        for _ in range(steps):
            lz.step(opfun)
        converge(p, min(d, lz.j - 1))
        th = np.linalg.eigvalsh(lz.T())
        mu_hat = th[min(d, lz.j) - 1]
        if (mu_ex is not None and mu_hat < mu_ex) or lz.j >= m_tar - m0 or lz.j >= room:
            break
    m_new = lz.j
    converge(max(1, opts.c_r * m_new), 0)
    th, P = np.linalg.eigh(lz.T())
    order = np.argsort(-th, kind="stable")
    th, P = th[order], P[:, order]
    st.lanczos_steps += lz.steps
    st.m_extended = m_new
    return np.hstack([Vini, lz.V @ P]), np.concatenate([Dini, th])


# --------------------------------------------------------------------------
def m_qr(M, F):
    """Column-scaled CholQR2 in the M inner product: Q^T M Q = I, span Q = span F."""
    nrm = np.sqrt(np.einsum("ij,ij->j", F, _apply_M(M, F)))
    Q = F / nrm
    for _ in range(2):
        G = _mdot(M, Q, Q)
        G = 0.5 * (G + G.T)
        R = np.linalg.cholesky(G).T  # upper
        Q = sla.solve_triangular(R, Q.T, trans="T", lower=False).T
    return Q


def refine(Ah, Mh, lev_l: _mmd.Level, Q0, D0, tol_rel, mu_re, eps_h, delta_h, opts: EigOpts,
           ctr: Counters, st: LevelStats):
    """Algorithm 5 (Eigenpair Refinement) from level l = h + 1 to level h."""
    m = Q0.shape[1]
    if m == 0:
        return Q0, D0
    # g_i = pcg(B^l, (U^l)^T M^h q_i, -, -, eps)
    R = _mmd.Ut_apply(lev_l, _apply_M(Mh, Q0))
    G = np.zeros_like(R)
    for i in range(m):
        G[:, i] = bsolve(Ah, lev_l, R[:, i], tol_rel, opts.max_cg_iter, ctr)
    F = Q0 * D0[None, :] + _mmd.U_apply(lev_l, G)
    Qprev = Q0
    D = D0.copy()
    stop = tol_rel / np.sqrt(1.0 + eps_h * delta_h)
    Q = Q0
    mh = m
    for it in range(1, opts.max_refine_iter + 1):
        Q = m_qr(Mh, F)
        W = _apply_M(Mh, Q)
        F = np.zeros_like(Q)
        for i in range(m):
            x, its, ok = fpcg(Ah, W[:, i], Mh, D[i] * Q[:, i], tol_rel, opts.max_cg_iter, ctr)
            F[:, i] = x
            ctr.refine_pcg_calls += 1
            ctr.refine_pcg_iters += its
            ctr.not_converged += 0 if ok else 1
        S = W.T @ F
        S = 0.5 * (S + S.T)
        D, P = np.linalg.eigh(S)
        order = np.argsort(-D, kind="stable")
        D, P = D[order], P[:, order]
        # renew m_h (keep mu_mh >= mu_re); keep a spectral gap to the end of the
        # window, mu_mh >= mu_ml * alpha / (1 + beta) (efficiency condition (ii), Section 6)
        mh = int(np.sum(D >= max(mu_re, D[-1] * opts.alpha / (1.0 + opts.beta))))
        Q = Q @ P
        F = F @ P
        st.refine_iters = it
        dQ = Q[:, :mh] - Qprev[:, :mh] @ _mdot(Mh, Qprev[:, :mh], Q[:, :mh])
        if np.linalg.norm(dQ) < stop:
            break
        Qprev = Q
    else:
        ctr.not_converged += 1
    st.m_refined = mh
    return Q[:, :mh], D[:mh]


# --------------------------------------------------------------------------
def auto_d(Nk: int, m_tar: int) -> int:
    return max(1, min(Nk // 10, m_tar // 10))


@dataclasses.dataclass
class EigResult:
    lam: np.ndarray
    V: np.ndarray
    counters: Counters
    levels: list
    mu1: float
    trace: list = dataclasses.field(default_factory=list)  # (k, mu values output on level k)


def eig_leftmost(D: _mmd.MMD, N: int, tol: float, opts: EigOpts | None = None) -> EigResult:
    """Algorithm 6 with the level-0 completion: N smallest eigenpairs of A."""
    opts = opts or EigOpts()
    ctr = Counters()
    K = D.K
    n = D.N(0)
    N = int(N)
    if N < 1 or N > n:
        raise ValueError("N out of range")
    lstats = []
    if opts.method == "irlm_cg":
        # Section 8's baseline: implicitly restarted Lanczos on A^{-1}, every
        # application by plain CG, no decomposition.  Algorithm 4 at level 0
        # from an empty basis with searching step d = N: one extension reaches
        # N columns and each restart of the final loop applies N exact shifts.
        st = LevelStats(0, n)
        A0 = D.A(0)
        Vh, Dh = extend(A0, None, np.zeros((n, 0)), np.zeros(0), 0.1 * tol,
                        lambda th, res: bool(np.all(res <= tol * np.abs(th))), None, N, N, opts, ctr, st, 1000)
        lstats.append(st)
        order = np.argsort(-Dh, kind="stable")[:N]
        return _finish(1.0 / Dh[order], Vh[:, order], ctr, lstats, 0.0)
    if not 0 <= opts.stop_level <= K:
        raise ValueError("stop_level out of range")
    last = opts.stop_level
    # coarsest level: (A^(K))^{-1} M^(K) x = mu x  <=>  A^(K) x = lambda M^(K) x
    AK = D.A(K).toarray()
    MK = np.eye(AK.shape[0]) if K == 0 else D.M(K).toarray()
    lam, Z = sla.eigh(AK, MK)
    mu = 1.0 / lam  # lambda ascending -> mu descending, columns of Z in the same order
    mu1 = float(mu[0])
    if K == 0:
        V, lam_out = Z[:, :N], 1.0 / mu[:N]
        return _finish(lam_out, V, ctr, lstats, mu1)
    epsK = D.levels[K - 1].eps
    if last == K:  # the coarse-level approximation (Section 7.2): the N largest mu of the pencil
        keep = min(len(mu), N)
    else:
        keep = min(int(np.sum(mu >= opts.beta * epsK)), N)
    Vh, Dh = Z[:, :keep], mu[:keep]
    lstats.append(LevelStats(K, D.N(K), m_extended=keep))
    trace = [(K, Dh.copy())]
    stream = 1000
    for k in range(K - 1, last - 1, -1):
        st = LevelStats(k, D.N(k))
        lev_l = D.levels[k]  # level k + 1 (its patches partition level k)
        Vh = lev_l.psi @ Vh  # Algorithm 6, coefficient transfer
        Ah, Mh = D.A(k), D.M(k)
        eps_l = lev_l.eps
        if k >= 1:
            eps_h = D.levels[k - 1].eps
            delta_h = D.levels[k - 1].delta
            tol_rel = float(np.clip(0.1 * eps_h / mu1, 1e-14, 0.1))
            eps_abs = 0.1 * eps_h
            res_ok = lambda th, res, e=eps_abs: bool(np.all(res <= e))
            mu_ex = opts.beta * eps_h if k > last else None  # the last level extends to N pairs
        else:
            eps_h, delta_h = 0.0, 0.0
            tol_rel = tol
            res_ok = lambda th, res: bool(np.all(res <= tol * np.abs(th)))
            mu_ex = None
        mu_re = opts.alpha * eps_l
        pcg_tol = 0.1 * tol_rel if k == 0 else tol_rel
        Vh, Dh = refine(Ah, Mh, lev_l, Vh, Dh, pcg_tol, mu_re, eps_h, delta_h, opts, ctr, st)
        d = opts.d if opts.d > 0 else auto_d(D.N(k), N)
        Vh, Dh = extend(Ah, Mh, Vh, Dh, pcg_tol, res_ok, mu_ex, d, N, opts, ctr, st, stream)
        stream += 1000
        lstats.append(st)
        trace.append((k, Dh.copy()))
    # a result on level s >= 1: V = Psi^(1) ... Psi^(s) V^(s) (Algorithm 6, last line)
    for j in range(last, 0, -1):
        Vh = D.levels[j - 1].psi @ Vh
    order = np.argsort(-Dh, kind="stable")[:N]
    res = _finish(1.0 / Dh[order], Vh[:, order], ctr, lstats, mu1)
    res.trace = trace
    return res


def _finish(lam, V, ctr, lstats, mu1):
    order = np.argsort(lam, kind="stable")
    lam, V = lam[order], V[:, order].copy()
    V /= np.linalg.norm(V, axis=0)
    for i in range(V.shape[1]):
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
    return EigResult(lam, V, ctr, lstats, mu1)


def residuals(A, lam, V):
    """||A v - lambda v||_2 per pair."""
    R = A @ V - V * lam[None, :]
    return np.linalg.norm(R, axis=0)
