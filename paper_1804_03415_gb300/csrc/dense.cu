// Small dense FP64 kernels of the eigensolver: the tridiagonal Lanczos
// matrix T (Algorithms 1-4), the implicit restart's shifted QR sweeps
// (Algorithm 2), the Rayleigh-Ritz matrix S and the M-QR Cholesky factor of
// the refinement (Algorithm 5) and the coarsest generalized eigenproblem
// (Algorithm 6, first step).
//
// GB300 has little FP64 throughput per SM and long FP64 latencies, so the
// classical sequential algorithms are restructured for parallel hardware:
//   * tridiagonal eigenvalues: Sturm-sequence bisection, one thread per
//     eigenvalue (Golub and Van Loan, Section 8.4);
//   * tridiagonal eigenvectors: implicit QL with Wilkinson shifts, the
//     rotations applied to the rows of Z in parallel, or to the last row
//     only when just the Ritz estimates are wanted;
//   * p explicitly shifted QR steps, one Givens sweep each: the p sweeps
//     move down the matrix together, sweep j three positions behind sweep
//     j-1, so one step of the schedule performs up to p independent
//     rotations; the rotations are recorded and applied to Q by many
//     blocks, one row of Q per thread;
//   * dense symmetric eigenproblems (Rayleigh-Ritz S, coarsest pencil):
//     cooperative two-sided Jacobi, round-robin pairs across blocks.
#include <cuda_runtime.h>

#include <mutex>

#include "dev_common.cuh"
#include "kernels.h"

namespace mmd {
namespace {

constexpr double kEps = 2.220446049250313e-16;

// ------------------------------------------------------------ bisection
__device__ int sturm_count(const double* d, const double* e2, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int k = 1; k < n; ++k) {
    q = d[k] - x - e2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;  // number of eigenvalues < x
}

__global__ void tri_bounds_kernel(const double* d, const double* e, int n, double* bounds, double* e2) {
  // bounds[0] = lo, bounds[1] = hi (Gershgorin), bounds[2] = pivmin
  __shared__ double slo[256], shi[256], smx[256];
  double lo = 1e300, hi = -1e300, mx = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double el = k > 0 ? fabs(e[k - 1]) : 0.0, er = k < n - 1 ? fabs(e[k]) : 0.0;
    lo = fmin(lo, d[k] - el - er);
    hi = fmax(hi, d[k] + el + er);
    mx = fmax(mx, fmax(fabs(d[k]), er));
    if (k < n - 1) e2[k] = e[k] * e[k];
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double span = fmax(shi[0] - slo[0], smx[0]);
    bounds[0] = slo[0] - 4 * kEps * span - 1e-300;
    bounds[1] = shi[0] + 4 * kEps * span + 1e-300;
    bounds[2] = fmax(smx[0] * kEps * kEps, 1e-300);
  }
}

__global__ void tri_bisect_kernel(const double* d, const double* e2, int n, const double* bounds, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lo = bounds[0], hi = bounds[1];
  const double pivmin = bounds[2];
  // find x with count(x) <= i < count(hi): the (i+1)-th smallest eigenvalue lies in [lo, hi)
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2 * kEps * fmax(fabs(lo), fabs(hi)) + pivmin || mid == lo || mid == hi) break;
    if (sturm_count(d, e2, n, mid, pivmin) > i)
      hi = mid;
    else
      lo = mid;
  }
  w[i] = 0.5 * (lo + hi);
}

// ------------------------------------------------------------ QR sweeps
// p explicitly shifted QR steps T - s_j I = Q_j R_j, T <- R_j Q_j + s_j I
// (Algorithm 2), each one Givens sweep down the tridiagonal.  With exact
// shifts the explicit step keeps the deflation that the implicit bulge chase
// loses in floating point.  One block; sd/se hold T in shared memory and
// shift j works at position k = step - 3 j, so shift j reads only entries
// that shift j - 1 has finished (d_{k+1} at position k + 1, e_{k+1} at k + 2).
// Per position: rotation k combines the partly reduced row k, (x, y) in
// columns (k, k+1), with row k+1 of T - s I; then
//   d'_k = c_{k-1} c_k R_kk + s_k R_{k,k+1} + s,   e'_{k-1} = s_{k-1} R_kk,
// and at k = n-2 also the last row (d'_{n-1}, e'_{n-2}).  Rotation (c, s) of
// step t for shift j is recorded at rc/rs[t * p + j] (c = 1, s = 0 when idle).
__global__ void tri_chase_kernel(double* d, double* e, int n, const double* sh, int p, double* rc, double* rs,
                                 int nsteps) {
  extern __shared__ double smem[];
  double* sd = smem;
  double* se = smem + n;
  double* sx = se + n;   // carried R row: diagonal candidate
  double* sy = sx + p;   //                superdiagonal candidate
  double* scp = sy + p;  // previous rotation of this shift
  double* ssp = scp + p;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    sd[k] = d[k];
    se[k] = (k < n - 1) ? e[k] : 0.0;
  }
  __syncthreads();
  for (int step = 0; step < nsteps; ++step) {
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const int k = step - 3 * j;
      double c = 1.0, s = 0.0;
      if (k >= 0 && k <= n - 2) {
        const double sj = sh[j];
        double x, y, cp, sp;
        if (k == 0) {
          x = sd[0] - sj;
          y = se[0];
          cp = 1.0;
          sp = 0.0;
        } else {
          x = sx[j];
          y = sy[j];
          cp = scp[j];
          sp = ssp[j];
        }
        const double ek = se[k], d1 = sd[k + 1] - sj, e1 = (k + 1 <= n - 2) ? se[k + 1] : 0.0;
        const double r = hypot(x, ek);
        if (r > 0) {
          c = x / r;
          s = ek / r;
        }
        const double rk1 = c * y + s * d1;
        const double xn = -s * y + c * d1;
        sd[k] = cp * c * r + s * rk1 + sj;
        if (k >= 1) se[k - 1] = sp * r;
        if (k == n - 2) {
          sd[n - 1] = c * xn + sj;
          se[n - 2] = s * xn;
        }
        sx[j] = xn;
        sy[j] = c * e1;
        scp[j] = c;
        ssp[j] = s;
      }
      rc[size_t(step) * p + j] = c;
      rs[size_t(step) * p + j] = s;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    d[k] = sd[k];
    if (k < n - 1) e[k] = se[k];
  }
}

// Q (starting from I) <- Q G_1 G_2 ... ; one row of Q per thread.
__global__ void tri_apply_rot_kernel(int n, int p, int nsteps, const double* rc, const double* rs, double* Q,
                                     int ldq) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  for (int k = 0; k < n; ++k) Q[row + size_t(k) * ldq] = (k == row) ? 1.0 : 0.0;
  for (int step = 0; step < nsteps; ++step) {
    int jlo = (step - (n - 2) + 2) / 3;
    if (jlo < 0) jlo = 0;
    int jhi = step / 3;
    if (jhi > p - 1) jhi = p - 1;
    for (int j = jlo; j <= jhi; ++j) {
      const int k = step - 3 * j;
      if (k < 0 || k > n - 2) continue;
      const double c = rc[size_t(step) * p + j], s = rs[size_t(step) * p + j];
      double* q0 = Q + row + size_t(k) * ldq;
      double* q1 = q0 + ldq;
      const double a = *q0, b = *q1;
      *q0 = c * a + s * b;
      *q1 = -s * a + c * b;
    }
  }
}

// ------------------------------------------------------------ implicit QR (tridiagonal)
// Symmetric tridiagonal eigen-decomposition by implicit QR steps with the
// Wilkinson shift, deflating at the bottom (Golub and Van Loan, Alg. 8.3.2
// and 8.3.3).  One block: thread 0 runs the scalar recurrence of one sweep
// and records its rotations in shared memory; then every thread applies the
// sweep to its rows of Z (Z <- Z G, full eigenvectors) when Z is given, and
// thread 0 applies it to the row vector zl = e_{n-1}^T Z (last components,
// the quantities of the Ritz estimate ||f|| |e_k^T y|) when zl is given.
// The sweep is one chain of dependent FP64 operations, so it keeps what the
// next rotation needs in registers (the running diagonal and off-diagonal
// entries, zl's active entry) and forms each rotation from one reciprocal
// square root; Z's rows carry their active entry in a register too, with the
// next entry loaded ahead.  On exit w holds the eigenvalues ascending (ties
// by position) and Z / zl are permuted alike.
__global__ void tri_ql_kernel(const double* d_in, const double* e_in, int n, double* w, double* Z, int ldz,
                              double* zl, int* status) {
  extern __shared__ double sm[];
  double* d = sm;
  double* e = d + n;
  double* rc = e + n;
  double* rs = rc + n;
  __shared__ int s_lo, s_hi, s_done, s_nswap;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    d[k] = d_in[k];
    e[k] = (k < n - 1) ? e_in[k] : 0.0;
  }
  if (Z)
    for (int64_t t = threadIdx.x; t < int64_t(n) * n; t += blockDim.x) {
      const int i = int(t % n), j = int(t / n);
      Z[i + size_t(j) * ldz] = (i == j) ? 1.0 : 0.0;
    }
  if (zl)
    for (int k = threadIdx.x; k < n; k += blockDim.x) zl[k] = (k == n - 1) ? 1.0 : 0.0;
  __syncthreads();
  int hi = n - 1, iters = 0;
  const int max_iters = 40 * n + 100;
  while (true) {
    if (threadIdx.x == 0) {
      s_done = 0;
      // deflate converged bottom entries
      while (hi > 0 && fabs(e[hi - 1]) <= kEps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
        e[hi - 1] = 0.0;
        --hi;
      }
      if (hi == 0 || iters >= max_iters) {
        s_done = 1;
        if (iters >= max_iters) atomicExch(status, (int)DEV_NOCONV);
      } else {
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > kEps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        const double dl = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double den = dl + (dl >= 0 ? 1.0 : -1.0) * hypot(dl, eh);
        const double mu = d[hi] - ((den != 0.0) ? eh * eh / den : 0.0);
        double a = d[lo], b = e[lo];  // d[k], e[k] as this rotation sees them
        double x = a - mu, z = b;
        double zk = zl ? zl[lo] : 0.0;
        for (int k = lo; k < hi; ++k) {
          const double dd = d[k + 1];
          const double e1 = (k < hi - 1) ? e[k + 1] : 0.0;
          const double z1 = zl ? zl[k + 1] : 0.0;
          const double r2 = fma(x, x, z * z);
          double c = 1.0, sn = 0.0, r = 0.0;
          if (r2 > 0.0) {
            const double inv = rsqrt(r2);
            c = x * inv;
            sn = z * inv;
            r = r2 * inv;
          }
          if (k > lo) e[k - 1] = r;
          const double cs = c * sn, cc = c * c, ss = sn * sn;
          d[k] = cc * a + 2 * cs * b + ss * dd;
          const double dk1 = ss * a - 2 * cs * b + cc * dd;
          const double ek = cs * (dd - a) + (cc - ss) * b;
          e[k] = ek;
          if (k < hi - 1) {
            z = sn * e1;
            b = c * e1;
          }
          x = ek;
          a = dk1;
          rc[k] = c;
          rs[k] = sn;
          if (zl) {
            zl[k] = c * zk + sn * z1;
            zk = -sn * zk + c * z1;
          }
        }
        d[hi] = a;
        if (zl) zl[hi] = zk;
        s_lo = lo;
        s_hi = hi;
        ++iters;
      }
    }
    __syncthreads();
    if (s_done) break;
    if (Z) {
      const int lo = s_lo, h2 = s_hi;
      for (int row = threadIdx.x; row < n; row += blockDim.x) {
        double* q = Z + row;
        double a0 = q[size_t(lo) * ldz], b0 = q[size_t(lo + 1) * ldz];
        for (int k = lo; k < h2; ++k) {
          const double bn = (k + 2 <= h2) ? q[size_t(k + 2) * ldz] : 0.0;
          q[size_t(k) * ldz] = rc[k] * a0 + rs[k] * b0;
          a0 = -rs[k] * a0 + rc[k] * b0;
          b0 = bn;
        }
        q[size_t(h2) * ldz] = a0;
      }
    }
    __syncthreads();
  }
  // sort ascending: every thread ranks its entries (ties by position), the
  // values and zl are scattered by rank, Z's columns permuted by the swaps
  // thread 0 derives from the ranks (each thread swaps within its own rows)
  int* rank = reinterpret_cast<int*>(rc);
  int* swaps = reinterpret_cast<int*>(rs);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = d[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (d[j] < v) || (d[j] == v && j < i);
    rank[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    w[rank[i]] = d[i];
    if (zl) e[rank[i]] = zl[i];
  }
  __syncthreads();
  if (zl)
    for (int i = threadIdx.x; i < n; i += blockDim.x) zl[i] = e[i];
  if (Z) {
    if (threadIdx.x == 0) {
      // column i moves to rank[i]: swap i with its destination until i holds its own column
      int ns = 0;
      for (int i = 0; i < n; ++i)
        while (rank[i] != i) {
          const int j = rank[i];
          swaps[2 * ns] = i;
          swaps[2 * ns + 1] = j;
          ++ns;
          rank[i] = rank[j];
          rank[j] = j;
        }
      s_nswap = ns;
    }
    __syncthreads();
    const int ns = s_nswap;
    for (int row = threadIdx.x; row < n; row += blockDim.x)
      for (int t = 0; t < ns; ++t) {
        double* p0 = Z + row + size_t(swaps[2 * t]) * ldz;
        double* p1 = Z + row + size_t(swaps[2 * t + 1]) * ldz;
        const double u = *p0;
        *p0 = *p1;
        *p1 = u;
      }
  }
}

// ------------------------------------------------------------ parallel Jacobi
// Two-sided cyclic Jacobi on a symmetric matrix (Golub and Van Loan, Section
// 8.5; parallel round-robin ordering, Section 8.5.5).  Jacobi keeps relative
// accuracy on graded matrices (Demmel and Veselic 1992), which the Rayleigh-
// Ritz matrices of the refinement are: nearly diagonal with Ritz values that
// span many orders of magnitude.  Cooperative launch; every round:
//   phase 1: one thread per pair (p, q) computes its rotation (c, s);
//   phase 2: one thread per 2x2 block {p,q} x {p',q'} applies both rotations
//            (S <- J^T S J), one thread per (row, pair) updates V <- V J.
// Pairs follow the round-robin tournament on m' = m rounded up to even
// (index m' - 1 is a dummy when m is odd).  Sweeps stop when every rotation
// of a sweep was skipped (|s_pq| <= 1e-15 sqrt(|s_pp s_qq|)) or after 30.
struct JacobiArgs {
  double* S;  // m x m, ld = m, destroyed (diagonal = eigenvalues)
  double* V;  // m x m, ld = m, eigenvectors
  int m;
  double* rc;  // m'/2
  double* rs;  // m'/2
  int* rot;    // [30]: rotations applied in each sweep (zeroed before launch)
  GridBarrier bar;
};

__device__ __forceinline__ void rr_pair(int round, int i, int mp, int& p, int& q) {
  // round-robin: player mp-1 fixed, others rotate
  const int a = (i == 0) ? mp - 1 : (round + i) % (mp - 1);
  const int b = (round + mp - 1 - i) % (mp - 1);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

__global__ void jacobi_kernel(JacobiArgs a) {
  grid_sync_init();
  const int m = a.m, mp = m + (m & 1), np = mp / 2;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nthr = int64_t(gridDim.x) * blockDim.x;
  double* S = a.S;
  double* V = a.V;
  for (int64_t t = tid; t < int64_t(m) * m; t += nthr) V[t] = ((t % m) == (t / m)) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (!grid_sync(a.bar)) return;
    for (int round = 0; round < mp - 1; ++round) {
      for (int64_t i = tid; i < np; i += nthr) {
        int p, q;
        rr_pair(round, (int)i, mp, p, q);
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = S[p + size_t(q) * m], app = S[p + size_t(p) * m], aqq = S[q + size_t(q) * m];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && apq != 0.0) {
            const double th = (aqq - app) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
            atomicAdd(a.rot + sweep, 1);
          }
        }
        a.rc[i] = c;
        a.rs[i] = s;
      }
      if (!grid_sync(a.bar)) return;
      // S <- J^T S J on 2x2 blocks, V <- V J
      for (int64_t t = tid; t < int64_t(np) * np; t += nthr) {
        const int i = int(t % np), j = int(t / np);
        int p, q, p2, q2;
        rr_pair(round, i, mp, p, q);
        rr_pair(round, j, mp, p2, q2);
        const double c1 = a.rc[i], s1 = a.rs[i], c2 = a.rc[j], s2 = a.rs[j];
        const bool qv = q < m, q2v = q2 < m;
        double x00 = S[p + size_t(p2) * m];
        double x01 = q2v ? S[p + size_t(q2) * m] : 0.0;
        double x10 = qv ? S[q + size_t(p2) * m] : 0.0;
        double x11 = (qv && q2v) ? S[q + size_t(q2) * m] : 0.0;
        // rows: [p; q] <- [c1 -s1; s1 c1]^T [p; q]
        const double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
        const double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
        // columns: [p2 q2] <- [p2 q2] [c2 s2; -s2 c2]
        S[p + size_t(p2) * m] = c2 * y00 - s2 * y01;
        if (q2v) S[p + size_t(q2) * m] = s2 * y00 + c2 * y01;
        if (qv) S[q + size_t(p2) * m] = c2 * y10 - s2 * y11;
        if (qv && q2v) S[q + size_t(q2) * m] = s2 * y10 + c2 * y11;
      }
      for (int64_t t = tid; t < int64_t(m) * np; t += nthr) {
        const int r = int(t % m), j = int(t / m);
        int p, q;
        rr_pair(round, j, mp, p, q);
        if (q >= m) continue;
        const double c = a.rc[j], s = a.rs[j];
        const double vp = V[r + size_t(p) * m], vq = V[r + size_t(q) * m];
        V[r + size_t(p) * m] = c * vp - s * vq;
        V[r + size_t(q) * m] = s * vp + c * vq;
      }
      if (!grid_sync(a.bar)) return;
    }
    if (!grid_sync(a.bar)) return;
    if (ld_acquire_int(a.rot + sweep) == 0) break;
  }
}

__global__ void permute_cols_kernel(const double* A, int lda, int64_t nrows, const int* perm, int ncols, double* B,
                                    int ldb) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < nrows * ncols;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t % nrows;
    const int c = int(t / nrows);
    B[r + int64_t(c) * ldb] = A[r + int64_t(perm[c]) * lda];
  }
}

// ------------------------------------------------------------ Cholesky family
__global__ void potrf_upper_kernel(double* A, int lda, int n, int* status) {
  // A = R^T R, R upper stored in the upper triangle; one block, right-looking
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double a = A[j + size_t(j) * lda];
      if (!(a > 0)) {
        atomicExch(status, (int)DEV_NOTSPD);
        piv = 1.0;
      } else {
        piv = sqrt(a);
      }
      A[j + size_t(j) * lda] = piv;
    }
    __syncthreads();
    const double pv = piv;
    for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) A[j + size_t(c) * lda] /= pv;
    __syncthreads();
    // trailing: A[r, c] -= R[j, r] R[j, c] for j < r <= c
    {
      const int w = n - j - 1;
      for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
        const int r = j + 1 + t % w, c = j + 1 + t / w;
        if (r <= c) A[r + size_t(c) * lda] -= A[j + size_t(r) * lda] * A[j + size_t(c) * lda];
      }
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    for (int r = c + 1; r < n; ++r) A[r + size_t(c) * lda] = 0.0;
}

// Rinv = R^{-1} (upper), one thread per column
__global__ void trinv_upper_kernel(const double* R, int ldr, int n, double* X, int ldx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double* x = X + size_t(j) * ldx;
  for (int i = n - 1; i >= 0; --i) {
    if (i > j) {
      x[i] = 0.0;
      continue;
    }
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = i + 1; k <= j; ++k) s -= R[i + size_t(k) * ldr] * x[k];
    x[i] = s / R[i + size_t(i) * ldr];
  }
}

__global__ void potrf_lower_kernel(double* A, int lda, int n, int* status) {
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double a = A[j + size_t(j) * lda];
      if (!(a > 0)) {
        atomicExch(status, (int)DEV_NOTSPD);
        piv = 1.0;
      } else {
        piv = sqrt(a);
      }
      A[j + size_t(j) * lda] = piv;
    }
    __syncthreads();
    const double pv = piv;
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) A[r + size_t(j) * lda] /= pv;
    __syncthreads();
    {
      const int w = n - j - 1;
      for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
        const int r = j + 1 + t % w, c = j + 1 + t / w;
        if (r >= c) A[r + size_t(c) * lda] -= A[r + size_t(j) * lda] * A[c + size_t(j) * lda];
      }
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    for (int r = 0; r < c; ++r) A[r + size_t(c) * lda] = 0.0;
}

__global__ void trsm_llnn_kernel(const double* L, int ldl, int n, double* B, int ldb, int nrhs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  double* b = B + size_t(c) * ldb;
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i + size_t(k) * ldl] * b[k];
    b[i] = s / L[i + size_t(i) * ldl];
  }
}
__global__ void trsm_lltn_kernel(const double* L, int ldl, int n, double* B, int ldb, int nrhs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  double* b = B + size_t(c) * ldb;
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[k + size_t(i) * ldl] * b[k];
    b[i] = s / L[i + size_t(i) * ldl];
  }
}

__global__ void transpose_kernel(const double* A, int lda, int n, double* B, int ldb) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(n) * n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t % n), j = int(t / n);
    B[j + size_t(i) * ldb] = A[i + size_t(j) * lda];
  }
}
__global__ void symmetrise_kernel(double* A, int lda, int n) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(n) * n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t % n), j = int(t / n);
    if (i > j) {
      const double v = 0.5 * (A[i + size_t(j) * lda] + A[j + size_t(i) * lda]);
      A[i + size_t(j) * lda] = v;
      A[j + size_t(i) * lda] = v;
    }
  }
}
__global__ void csr_dense_kernel(const int32_t* rp, const int32_t* ci, const double* va, int n, double* D, int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < n; ++k) D[i + size_t(k) * ldd] = 0.0;
  for (int32_t k = rp[i]; k < rp[i + 1]; ++k) D[i + size_t(ci[k]) * ldd] = va[k];
}
inline int g1(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// scratch layout owned by the caller: see Workspace (api.cu).
struct TriScratch {
  double* bounds;  // 4
  double* e2;      // n
  int* cstart;     // n + 1
  int* ncl;        // 1
  double* work;    // 5 n^2
  int* iwork;      // n^2
};
// one per host thread: concurrent solves (eig_leftmost_batched) use their own
static thread_local TriScratch g_tri = {};

void set_tri_scratch(double* bounds, double* e2, int* cstart, int* ncl, double* work, int* iwork) {
  g_tri = {bounds, e2, cstart, ncl, work, iwork};
}

void k_tri_eigvals(const double* d, const double* e, int n, double* w, cudaStream_t st) {
  tri_bounds_kernel<<<1, 256, 0, st>>>(d, e, n, g_tri.bounds, g_tri.e2);
  tri_bisect_kernel<<<(n + 63) / 64, 64, 0, st>>>(d, g_tri.e2, n, g_tri.bounds, w);
}

void k_tri_ql(const double* d, const double* e, int n, double* w, double* Z, int ldz, double* zl, int* status,
              cudaStream_t st) {
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(tri_ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const size_t smem = sizeof(double) * 4 * size_t(n);
  tri_ql_kernel<<<1, 512, smem, st>>>(d, e, n, w, Z, ldz, zl, status);
}

void k_tri_qr_sweeps(double* d, double* e, int n, const double* sh, int p, double* Q, int ldq, cudaStream_t st) {
  const int nsteps = (n - 1) + 3 * (p - 1);
  double* rc = g_tri.work;
  double* rs = g_tri.work + size_t(nsteps) * p;
  const size_t smem = sizeof(double) * (2 * size_t(n) + 4 * size_t(p));
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(tri_chase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  tri_chase_kernel<<<1, 512, smem, st>>>(d, e, n, sh, p, rc, rs, nsteps);
  tri_apply_rot_kernel<<<(n + 7) / 8, 8, 0, st>>>(n, p, nsteps, rc, rs, Q, ldq);
}

static thread_local int g_coop_cap = 0;
void set_coop_grid_cap(int blocks) { g_coop_cap = blocks; }
int coop_grid_cap() { return g_coop_cap; }

int jacobi_max_grid() {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, jacobi_kernel, 256, 0);
  return nb * nsm;
}

cudaError_t k_syev_jacobi(double* S, int m, double* V, double* work, int* iwork, GridBarrier bar, cudaStream_t st) {
  JacobiArgs a;
  a.S = S;
  a.V = V;
  a.m = m;
  a.rc = work;
  a.rs = work + (m / 2 + 1);
  a.rot = iwork;
  a.bar = bar;
  cudaMemsetAsync(iwork, 0, 30 * sizeof(int), st);
  cudaMemsetAsync(bar.count, 0, sizeof(unsigned), st);
  static const int grid = jacobi_max_grid();  // thread-safe one-time initialisation
  int g = grid;
  if (coop_grid_cap() > 0 && g > coop_grid_cap()) g = coop_grid_cap();
  const int64_t need = (int64_t(m + 1) * (m + 1) / 4 + 255) / 256;
  if (g > need) g = (int)need;
  if (g < 1) g = 1;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(g), dim3(256), args, 0, st);
}

void k_permute_cols(const double* A, int lda, int64_t nrows, const int* perm, int ncols, double* B, int ldb,
                    cudaStream_t st) {
  int64_t b = (nrows * ncols + 255) / 256;
  if (b > 8192) b = 8192;
  if (b < 1) b = 1;
  permute_cols_kernel<<<(int)b, 256, 0, st>>>(A, lda, nrows, perm, ncols, B, ldb);
}

void k_potrf_upper(double* A, int lda, int n, int* dev_status, cudaStream_t st) {
  potrf_upper_kernel<<<1, 1024, 0, st>>>(A, lda, n, dev_status);
}
void k_trinv_upper(const double* R, int ldr, int n, double* Rinv, int ldri, cudaStream_t st) {
  trinv_upper_kernel<<<(n + 63) / 64, 64, 0, st>>>(R, ldr, n, Rinv, ldri);
}
void k_potrf_lower(double* A, int lda, int n, int* dev_status, cudaStream_t st) {
  potrf_lower_kernel<<<1, 1024, 0, st>>>(A, lda, n, dev_status);
}
void k_trsm_llnn(const double* L, int ldl, int n, double* B, int ldb, int nrhs, cudaStream_t st) {
  trsm_llnn_kernel<<<(nrhs + 63) / 64, 64, 0, st>>>(L, ldl, n, B, ldb, nrhs);
}
void k_trsm_lltn(const double* L, int ldl, int n, double* B, int ldb, int nrhs, cudaStream_t st) {
  trsm_lltn_kernel<<<(nrhs + 63) / 64, 64, 0, st>>>(L, ldl, n, B, ldb, nrhs);
}
void k_transpose_sq(const double* A, int lda, int n, double* B, int ldb, cudaStream_t st) {
  transpose_kernel<<<g1(int64_t(n) * n, 256), 256, 0, st>>>(A, lda, n, B, ldb);
}
void k_symmetrise(double* A, int lda, int n, cudaStream_t st) {
  symmetrise_kernel<<<g1(int64_t(n) * n, 256), 256, 0, st>>>(A, lda, n);
}
void k_csr_to_dense(const int32_t* rp, const int32_t* ci, const double* va, int n, double* D, int ldd,
                    cudaStream_t st) {
  csr_dense_kernel<<<(n + 127) / 128, 128, 0, st>>>(rp, ci, va, n, D, ldd);
}
}  // namespace mmd
