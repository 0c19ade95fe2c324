// Persistent CG / flexible-PCG kernel: the inner loop of Operator OP
// (Section 4: y = pcg(A^(k), M^(k) x, M^(k), 0, eps), with M^(k)^{-1} applied
// by an inner CG to 0.1 eps) and of the two solves of the Eigenpair
// Refinement (Algorithm 5: CG on B^(l) = U^T A U and the warm-started PCG).
//
// One cooperative launch (one 1024-thread block per SM) runs a whole solve for
// m <= MT right-hand sides (column-major, leading dimension ld).  Scalars never
// leave the device: each block writes its partial sums, a bounded grid barrier
// follows, and every block then reduces the same partials in the same order,
// so all blocks take identical decisions.
//
// GB300 retires about one FP64 warp-instruction per 16 SM cycles, so the
// kernel is organised to issue as few FP64 instructions as the arithmetic
// needs: the matrices are in SELL-32 (one row per lane, one FMA per stored
// entry, no shuffle reductions inside a row), and a block reduction is one
// pass of warp 0 over the threads' partials in shared memory.
//
// Precision: T = double (every step FP64) or T = float (matrix values,
// vectors and per-thread sums in FP32; block sums and scalars in FP64).  The
// FP32 instance is the inner solver of the mixed mode, wrapped by the driver
// in FP64 iterative refinement (FP64 residual b - A x, FP32 correction).
//
// Modes
//   0  CG on A (M = I; the paper's pcg(A, b, -, x0, eps)) in the
//      Chronopoulos-Gear form: one fused reduction, two barriers/iteration.
//   1  flexible PCG on A with preconditioner M applied by an inner CG;
//      beta = z+^T (r+ - r) / (r^T z)  (Golub and Ye, 1999), computed as
//      -alpha z+^T q / (r^T z) since r+ - r = -alpha q.
//   2  CG on P A P with P = I - Phi Phi^T applied segment by segment.  Since
//      U of Section 2.3 has orthonormal columns and U U^T = P on each patch,
//      this is CG on B = U^T A U in the coordinates U g (same iterates); the
//      solution returned is x = U g.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "kernels.h"

namespace mmd {

namespace {

constexpr int kThreads = 1024;

template <int MT>
struct Sh {
  double part[kThreads + 1];
  double bn[MT], rz[MT], rr[MT], alpha[MT], val[MT], val2[MT];
  double irr[MT], irn0[MT], ia[MT];
  int act[MT], iact[MT];
  long long it[MT], iit[MT];
};

// Block sum: every thread stores its partial; warp 0 adds 32 per lane and
// shuffles (37 FP64 warp-instructions per block instead of a shuffle tree in
// all 32 warps).  Result in part[kThreads].
__device__ __forceinline__ void block_reduce_to(double v, double* part) {
  part[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < kThreads; i += 32) t += part[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) part[kThreads] = t;
  }
  __syncthreads();
}

// partial sums red[slot][c][block] -> dst[c] (shared) in every block; one warp
template <int MT>
__device__ void reduce_slot(const double* red, int slot, int m, double* dst) {
  const int G = gridDim.x;
  if (threadIdx.x < 32) {
    for (int c = 0; c < m; ++c) {
      const double* p = red + (size_t(slot) * MT + c) * G;
      double t = 0.0;
      for (int b = threadIdx.x; b < G; b += 32) t += p[b];
      t = warp_sum(t);
      if (threadIdx.x == 0) dst[c] = t;
    }
  }
  __syncthreads();
}

template <int MT, typename T>
__device__ void write_partials(double* red, int slot, int m, const T* acc, Sh<MT>& s) {
  for (int c = 0; c < m; ++c) {
    block_reduce_to((double)acc[c], s.part);
    if (threadIdx.x == 0) red[(size_t(slot) * MT + c) * gridDim.x + blockIdx.x] = s.part[kThreads];
    __syncthreads();
  }
}

// Y(:,c) = A X(:,c) for columns with mask[c] (SELL-32, one row per lane);
// optionally dacc[c] += W(row,c) * Y(row,c).  The entry loop is unrolled by 4
// so the loads of four entries are in flight before their gathers.
template <int MT, typename T>
__device__ __forceinline__ void spmv_cols(const Sell& A, const T* __restrict__ X, T* __restrict__ Y, int64_t ld,
                                          int m, const int* mask, const T* __restrict__ W, T* dacc) {
  const T* __restrict__ vals = (sizeof(T) == 8) ? (const T*)A.val : (const T*)A.val32;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  int msk[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) msk[c] = (c < m) && mask[c];
  for (int64_t sl = gw; sl < A.nslices; sl += nw) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    T acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    int32_t k = 0;
    for (; k + 4 <= len; k += 4) {
      T a[4];
      int64_t j[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = vals[base + (k + u) * 32];
        j[u] = A.col[base + (k + u) * 32];
      }
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) {
          T xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) xv[u] = X[j[u] + c * ld];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[c] = fma(a[u], xv[u], acc[c]);
        }
    }
    for (; k < len; ++k) {
      const T a = vals[base + k * 32];
      const int64_t j = A.col[base + k * 32];
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) acc[c] = fma(a, X[j + c * ld], acc[c]);
    }
    if (row >= 0) {
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) {
          Y[row + c * ld] = acc[c];
          if (W) dacc[c] = fma(W[row + c * ld], acc[c], dacc[c]);
        }
    }
  }
}

template <int MT, typename T>
__device__ bool inner_cg(const SolverArgs& a, Sh<MT>& s, int64_t tid, int64_t nthr) {
  // z = M^{-1} r for active columns, CG to relative residual itol (zero start).
  T* const r = (T*)a.r;
  T* const z = (T*)a.z;
  T* const ir = (T*)a.ir;
  T* const ip = (T*)a.ip;
  T* const iq = (T*)a.iq;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  T acc[MT];
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    s.iact[c] = s.act[c] && s.rr[c] > 0.0;
    s.irr[c] = s.rr[c];
    s.irn0[c] = sqrt(s.rr[c]);
    s.iit[c] = 0;
  }
  __syncthreads();
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c)
      if (s.act[c]) {
        const T rv = r[i + c * ld];
        z[i + c * ld] = T(0);
        ir[i + c * ld] = rv;
        ip[i + c * ld] = rv;
      }
  if (!grid_sync(a.bar)) return false;
  for (int j = 1; j <= a.imaxit; ++j) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.iact[c];
    if (!any) break;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T>(a.M, ip, iq, ld, m, s.iact, ip, acc);
    write_partials<MT, T>(a.red, 2, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 2, m, s.val);
    if (threadIdx.x < m) s.ia[threadIdx.x] = s.iact[threadIdx.x] ? s.irr[threadIdx.x] / s.val[threadIdx.x] : 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.iact[c]) {
          const int64_t o = i + c * ld;
          const T al = (T)s.ia[c];
          z[o] = fma(al, ip[o], z[o]);
          const T rv = fma(-al, iq[o], ir[o]);
          ir[o] = rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    write_partials<MT, T>(a.red, 3, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 3, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.iact[c]) {
        s.iit[c] = j;
        const double rn = s.val[c];
        s.ia[c] = rn / s.irr[c];  // beta
        s.irr[c] = rn;
        if (sqrt(rn) <= a.itol * s.irn0[c]) s.iact[c] = 0;
      }
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.iact[c]) {
          const int64_t o = i + c * ld;
          ip[o] = fma((T)s.ia[c], ip[o], ir[o]);
        }
    if (!grid_sync(a.bar)) return false;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long t = 0;
    for (int c = 0; c < m; ++c) t += s.iit[c];
    *a.in_out += t;
  }
  return true;
}

// Mode 0: CG in the Chronopoulos-Gear form (one fused reduction of r^T r and
// r^T A r per iteration, so two grid barriers instead of three); same
// iterates as Hestenes-Stiefel CG in exact arithmetic.
// On entry r = b - A x0 is complete and s.rr = r^T r, s.act, s.bn are set.
template <int MT, typename T>
__device__ bool cgcg(const SolverArgs& a, Sh<MT>& s, int64_t tid, int64_t nthr) {
  T* const r = (T*)a.r;
  T* const p = (T*)a.p;
  T* const x = (T*)a.x;
  T* const w = (T*)a.z;
  T* const sv = (T*)a.q;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  T acc[MT];
  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.act[c];
    if (!any) break;
    // w = A r, delta = r^T w
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T>(a.A, r, w, ld, m, s.act, r, acc);
    write_partials<MT, T>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 0, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        const double g = s.rr[c], dl = s.val[c];
        double be = 0.0, den = dl;
        if (it > 1) {
          be = g / s.rz[c];
          den = dl - be * g / s.alpha[c];
        }
        if (!(den > 0.0)) {
          s.act[c] = 0;
          if (blockIdx.x == 0) atomicExch(a.bar.status, (int)DEV_NOTSPD);
        }
        s.rz[c] = g;
        s.alpha[c] = g / den;
        s.val2[c] = be;
      }
    }
    __syncthreads();
    // p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s, gamma = r^T r
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    const bool first = (it == 1);
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.act[c]) {
          const int64_t o = i + c * ld;
          const T be = (T)s.val2[c], al = (T)s.alpha[c];
          const T rv0 = r[o];
          const T pv = first ? rv0 : fma(be, p[o], rv0);
          const T svv = first ? w[o] : fma(be, sv[o], w[o]);
          p[o] = pv;
          sv[o] = svv;
          x[o] = fma(al, pv, x[o]);
          const T rv = fma(-al, svv, rv0);
          r[o] = rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    write_partials<MT, T>(a.red, 1, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 1, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        s.it[c] = it;
        s.rr[c] = s.val[c];
        if (sqrt(s.val[c]) <= a.tol * s.bn[c]) s.act[c] = 0;
      }
    }
    __syncthreads();
  }
  return true;
}

// FP64 residual of the reliable update: rr32 = (float)(b64 - A x64), partial
// sums of its square; FP64 SELL SpMV (matrix values in FP64).
template <int MT>
__device__ void reliable_residual(const SolverArgs& a, const int* mask, float* r32, double* acc) {
  const Sell& A = a.A;
  const int m = a.m;
  const int64_t ld = a.ld;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t sl = gw; sl < A.nslices; sl += nw) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    double ax[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) ax[c] = 0.0;
    for (int32_t k = 0; k < len; ++k) {
      const double v = A.val[base + k * 32];
      const int64_t j = A.col[base + k * 32];
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (c < m && mask[c]) ax[c] = fma(v, a.x64[j + c * ld], ax[c]);
    }
    if (row >= 0) {
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (c < m && mask[c]) {
          const double rv = a.b64[row + c * ld] - ax[c];
          r32[row + c * ld] = (float)rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    }
  }
}

// Mode 0, FP32 with FP64 reliable updates (residual replacement): the CG
// recurrences run in FP32, x accumulates in FP64, and whenever the FP32
// residual has dropped by 100x since the last replacement -- and before
// convergence is accepted -- r is replaced by the FP64 residual b - A x.
// The Krylov recurrence is kept (no restart), so the iteration count stays
// close to the FP64 one while the SpMV and vector traffic is FP32.
template <int MT>
__device__ bool cgcg_rel(const SolverArgs& a, Sh<MT>& s, int64_t tid, int64_t nthr) {
  float* const r = (float*)a.r;
  float* const p = (float*)a.p;
  float* const w = (float*)a.z;
  float* const sv = (float*)a.q;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  float acc[MT];
  double dacc[MT];
  // initial residual in FP64 (x64 = x0 or 0)
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) {
    all1[c] = 1;
    dacc[c] = 0.0;
  }
  if (!a.x0)
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c) a.x64[i + c * ld] = 0.0;
  if (!grid_sync(a.bar)) return false;
  reliable_residual<MT>(a, all1, r, dacc);
  write_partials<MT, double>(a.red, 1, m, dacc, s);
#pragma unroll
  for (int c = 0; c < MT; ++c) dacc[c] = 0.0;
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c) dacc[c] = fma(a.b64[i + c * ld], a.b64[i + c * ld], dacc[c]);
  write_partials<MT, double>(a.red, 0, m, dacc, s);
  if (!grid_sync(a.bar)) return false;
  reduce_slot<MT>(a.red, 0, m, s.bn);
  reduce_slot<MT>(a.red, 1, m, s.rr);
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    s.bn[c] = sqrt(s.bn[c]);
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.rr[c]) <= a.tol * s.bn[c]);
    s.it[c] = 0;
    s.irn0[c] = sqrt(s.rr[c]);  // norm at the last replacement
  }
  __syncthreads();
  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.act[c];
    if (!any) break;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0f;
    spmv_cols<MT, float>(a.A, r, w, ld, m, s.act, r, acc);
    write_partials<MT, float>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 0, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        const double g = s.rr[c], dl = s.val[c];
        double be = 0.0, den = dl;
        if (it > 1) {
          be = g / s.rz[c];
          den = dl - be * g / s.alpha[c];
        }
        if (!(den > 0.0)) {
          s.act[c] = 0;
          if (blockIdx.x == 0) atomicExch(a.bar.status, (int)DEV_NOTSPD);
        }
        s.rz[c] = g;
        s.alpha[c] = g / den;
        s.val2[c] = be;
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0f;
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.act[c]) {
          const int64_t o = i + c * ld;
          const bool fresh = (it == 1);
          const float be = (float)s.val2[c], al = (float)s.alpha[c];
          const float rv0 = r[o];
          const float pv = fresh ? rv0 : fmaf(be, p[o], rv0);
          const float svv = fresh ? w[o] : fmaf(be, sv[o], w[o]);
          p[o] = pv;
          sv[o] = svv;
          a.x64[o] = fma(s.alpha[c], (double)pv, a.x64[o]);
          const float rv = fmaf(-al, svv, rv0);
          r[o] = rv;
          acc[c] = fmaf(rv, rv, acc[c]);
        }
    write_partials<MT, float>(a.red, 1, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 1, m, s.val);
    // replacement needed?  (FP32 residual 100x below the last replaced one, or converged)
    int need = 0;
    for (int c = 0; c < m; ++c)
      if (s.act[c] && (sqrt(s.val[c]) <= 0.01 * s.irn0[c] || sqrt(s.val[c]) <= a.tol * s.bn[c])) need = 1;
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        s.it[c] = it;
        s.rr[c] = s.val[c];
      }
    }
    __syncthreads();
    if (need) {
      int msk[MT];
#pragma unroll
      for (int c = 0; c < MT; ++c) {
        msk[c] = (c < m) && s.act[c];
        dacc[c] = 0.0;
      }
      reliable_residual<MT>(a, msk, r, dacc);  // x64 is complete: the barrier above
      write_partials<MT, double>(a.red, 2, m, dacc, s);
      if (!grid_sync(a.bar)) return false;
      reduce_slot<MT>(a.red, 2, m, s.val2);
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c]) {
          s.rr[c] = s.val2[c];
          s.irn0[c] = sqrt(s.val2[c]);
          if (sqrt(s.val2[c]) <= a.tol * s.bn[c]) s.act[c] = 0;
        }
      }
      __syncthreads();
    }
  }
  return true;
}

template <int MT, typename T>
__global__ void __launch_bounds__(kThreads, 1) solve_kernel(SolverArgs a) {
  __shared__ Sh<MT> s;
  grid_sync_init();
  T* const b = (T*)a.b;
  T* const x = (T*)a.x;
  T* const r = (T*)a.r;
  T* const p = (T*)a.p;
  T* const q = (T*)a.q;
  T* const z = (T*)a.z;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  if constexpr (sizeof(T) == 4) {
    if (a.mode == 0 && a.b64) {
      if (!cgcg_rel<MT>(a, s, tid, nthr)) return;
      if (blockIdx.x == 0 && threadIdx.x < m) {
        a.it_out[threadIdx.x] = s.it[threadIdx.x];
        a.conv[threadIdx.x] = s.act[threadIdx.x] ? 0 : 1;
      }
      return;
    }
  }
  T acc[MT], acc2[MT];
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) all1[c] = 1;
  // ---- set-up: r = b - A x0 (or b), norms
  if (a.x0) {
    spmv_cols<MT, T>(a.A, x, q, ld, m, all1, nullptr, nullptr);
    if (!grid_sync(a.bar)) return;
  }
#pragma unroll
  for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = T(0);
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c) {
      const int64_t o = i + c * ld;
      const T bv = b[o];
      T rv = bv;
      if (a.x0) rv -= q[o];
      else x[o] = T(0);
      r[o] = rv;
      acc[c] = fma(bv, bv, acc[c]);
      acc2[c] = fma(rv, rv, acc2[c]);
    }
  write_partials<MT, T>(a.red, 0, m, acc, s);
  write_partials<MT, T>(a.red, 1, m, acc2, s);
  if (!grid_sync(a.bar)) return;
  reduce_slot<MT>(a.red, 0, m, s.bn);
  reduce_slot<MT>(a.red, 1, m, s.rr);
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    s.bn[c] = sqrt(s.bn[c]);
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.rr[c]) <= a.tol * s.bn[c]);
    s.it[c] = 0;
  }
  __syncthreads();
  for (int64_t i = tid; i < n; i += nthr)  // zero right-hand sides give x = 0
    for (int c = 0; c < m; ++c)
      if (s.bn[c] == 0.0) x[i + c * ld] = T(0);
  if (a.mode == 0) {
    if (!cgcg<MT, T>(a, s, tid, nthr)) return;
    if (blockIdx.x == 0 && threadIdx.x < m) {
      a.it_out[threadIdx.x] = s.it[threadIdx.x];
      a.conv[threadIdx.x] = s.act[threadIdx.x] ? 0 : 1;
    }
    return;
  }
  T* zv = r;
  if (a.mode == 1) {
    if (!inner_cg<MT, T>(a, s, tid, nthr)) return;
    zv = z;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.act[c]) acc[c] = fma(r[i + c * ld], z[i + c * ld], acc[c]);
    write_partials<MT, T>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 0, m, s.rz);
  } else {
    if (threadIdx.x < m) s.rz[threadIdx.x] = s.rr[threadIdx.x];
    __syncthreads();
  }
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c)
      if (s.act[c]) p[i + c * ld] = zv[i + c * ld];
  if (!grid_sync(a.bar)) return;

  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.act[c];
    if (!any) break;
    // q = A p, p^T q
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T>(a.A, p, q, ld, m, s.act, p, acc);
    write_partials<MT, T>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 0, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        if (!(s.val[c] > 0.0)) {  // p^T A p <= 0: not SPD (or p = 0)
          s.act[c] = 0;
          s.alpha[c] = 0.0;
          if (blockIdx.x == 0) atomicExch(a.bar.status, (int)DEV_NOTSPD);
        } else {
          s.alpha[c] = s.rz[c] / s.val[c];
        }
      }
    }
    __syncthreads();
    // x += alpha p, r -= alpha q (mode 2: q projected per segment), r^T r
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    if (a.mode == 2) {
      for (int64_t sg = tid; sg < a.nseg; sg += nthr) {
        const int32_t s0 = a.seg_ptr[sg], s1 = a.seg_ptr[sg + 1];
        for (int c = 0; c < m; ++c) {
          if (!s.act[c]) continue;
          const T al = (T)s.alpha[c];
          T t = T(0);
          for (int32_t i = s0; i < s1; ++i) t = fma((T)a.phi[i], q[i + c * ld], t);
          for (int32_t i = s0; i < s1; ++i) {
            const int64_t o = i + c * ld;
            const T qv = fma(-(T)a.phi[i], t, q[o]);
            x[o] = fma(al, p[o], x[o]);
            const T rv = fma(-al, qv, r[o]);
            r[o] = rv;
            acc[c] = fma(rv, rv, acc[c]);
          }
        }
      }
    } else {
      for (int64_t i = tid; i < n; i += nthr)
        for (int c = 0; c < m; ++c)
          if (s.act[c]) {
            const int64_t o = i + c * ld;
            const T al = (T)s.alpha[c];
            x[o] = fma(al, p[o], x[o]);
            const T rv = fma(-al, q[o], r[o]);
            r[o] = rv;
            acc[c] = fma(rv, rv, acc[c]);
          }
    }
    write_partials<MT, T>(a.red, 1, m, acc, s);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 1, m, s.val2);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        s.it[c] = it;
        if (sqrt(s.val2[c]) <= a.tol * s.bn[c]) s.act[c] = -1;  // converged this iteration
      }
    }
    __syncthreads();
    if (a.mode == 1) {
      // columns that just converged (-1) need no preconditioning
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c] < 0) s.act[c] = 0;
        s.rr[c] = s.val2[c];
      }
      __syncthreads();
      if (!inner_cg<MT, T>(a, s, tid, nthr)) return;
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = T(0);
      for (int64_t i = tid; i < n; i += nthr)
        for (int c = 0; c < m; ++c)
          if (s.act[c]) {
            const int64_t o = i + c * ld;
            acc[c] = fma(r[o], z[o], acc[c]);
            acc2[c] = fma(z[o], q[o], acc2[c]);
          }
      write_partials<MT, T>(a.red, 0, m, acc, s);
      write_partials<MT, T>(a.red, 1, m, acc2, s);
      if (!grid_sync(a.bar)) return;
      reduce_slot<MT>(a.red, 0, m, s.val);
      reduce_slot<MT>(a.red, 1, m, s.val2);
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c]) {
          s.alpha[c] = -s.alpha[c] * s.val2[c] / s.rz[c];  // beta
          s.rz[c] = s.val[c];
        }
      }
    } else {
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c] < 0) s.act[c] = 0;
        if (s.act[c]) {
          s.alpha[c] = s.val2[c] / s.rz[c];  // beta
          s.rz[c] = s.val2[c];
        }
      }
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.act[c]) {
          const int64_t o = i + c * ld;
          p[o] = fma((T)s.alpha[c], p[o], zv[o]);
        }
    if (!grid_sync(a.bar)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x < m) {
    const int c = threadIdx.x;
    a.it_out[c] = s.it[c];
    a.conv[c] = s.act[c] ? 0 : 1;
  }
}

template <int MT, typename T>
int max_blocks_for() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<MT, T>, kThreads, 0);
  return nb;
}

template <int MT, typename T>
cudaError_t launch_tpl(const SolverArgs& a, int grid, cudaStream_t st) {
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)solve_kernel<MT, T>, dim3(grid), dim3(kThreads), args, 0, st);
}

}  // namespace

int solver_threads() { return kThreads; }

// One block per SM (the reductions read one partial per block, <= 1024).
int solver_max_grid(int mt, int num_sms) {
  const int nb = (mt == 1) ? std::min(max_blocks_for<1, double>(), max_blocks_for<1, float>())
                           : std::min(max_blocks_for<8, double>(), max_blocks_for<8, float>());
  const int g = (nb >= 1) ? num_sms : 0;
  return g > kThreads ? kThreads : g;
}

cudaError_t launch_solver(const SolverArgs& a, int mt, int grid, cudaStream_t st) {
  if (a.fp32) {
    if (mt == 1) return launch_tpl<1, float>(a, grid, st);
    if (mt == 8) return launch_tpl<8, float>(a, grid, st);
  } else {
    if (mt == 1) return launch_tpl<1, double>(a, grid, st);
    if (mt == 8) return launch_tpl<8, double>(a, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mmd
