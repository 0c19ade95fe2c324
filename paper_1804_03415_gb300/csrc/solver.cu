// Persistent CG / flexible-PCG kernel: the inner loop of Operator OP
// (Section 4: y = pcg(A^(k), M^(k) x, M^(k), 0, eps), with M^(k)^{-1} applied
// by an inner CG to 0.1 eps) and of the two solves of the Eigenpair
// Refinement (Algorithm 5: CG on B^(l) = U^T A U and the warm-started PCG).
//
// One cooperative launch (one 1024-thread block per SM) runs a whole solve
// for m <= MT right-hand sides (column-major,
// leading dimension ld).  Scalars never leave the device: each block writes its partial sums, a bounded grid barrier
// follows, and every block then reduces the same partials in the same order,
// so all blocks take identical decisions.
//
// GB300 retires about one FP64 warp-instruction per 16 SM cycles, so the
// kernel is organised to issue as few FP64 instructions as the arithmetic
// needs: the matrices are in SELL-32 (one row per lane, one FMA per stored
// entry, no shuffle reductions inside a row), and a block reduction adds the
// threads' partials from shared memory with all lanes busy, the columns (or
// quarters of one column) spread over the SM's sub-partitions.
//
// Precision: T = double (every step FP64) or T = float (matrix values,
// vectors and per-thread sums in FP32; block sums and scalars in FP64).  The
// FP32 instance is the inner solver of the mixed mode, wrapped in driver.cu
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
#include <mutex>

#include "dev_common.cuh"
#include "kernels.h"

namespace mmd {

namespace {

// Threads per block (one block per SM).  Tiles are one or four columns
// wide: four accumulators and their gathers fit the 64 registers a thread
// gets at 1024 threads per SM (an eight-column tile needed 512-thread blocks
// for its registers and cost 3% more per column-iteration).
template <int MT>
__host__ __device__ constexpr int threads_for() {
  return 1024;
}
constexpr int kMaxThreads = 1024;

template <int MT>
struct Sh {
  double quart[2 * MT * 4];  // block reduction: per-warp sums, up to 4 warps per value
  double bn[MT], rz[MT], rr[MT], alpha[MT], val[MT], val2[MT];
  double irr[MT], irn0[MT], ia[MT];
  int act[MT], iact[MT];
  int due[MT], stag[MT];  // reliable updates: replacement due / no progress since the last one
  int ok[MT];             // reliable updates: stopped with the true residual below tol
  long long it[MT], iit[MT];
};

// Work split: block b owns the contiguous share [n b / G, n (b + 1) / G) of
// the rows (or segments, or SELL slices); its threads (warps, for slices)
// stride through it.  Every block gets within one unit of the same amount,
// where a grid-wide stride gave the first blocks a whole extra round (n =
// 200k rows on 152 x 1024 threads: 2048 rows on some SMs, 1024 on others).
__device__ __forceinline__ int64_t share_lo(int64_t n) { return n * blockIdx.x / gridDim.x; }
__device__ __forceinline__ int64_t share_hi(int64_t n) { return n * (blockIdx.x + 1) / gridDim.x; }
#define FOR_BLOCK_SHARE(i, n) \
  for (int64_t i = share_lo(n) + threadIdx.x, i##_end = share_hi(n); i < i##_end; i += blockDim.x)
#define FOR_BLOCK_SLICES(sl, ns) \
  for (int64_t sl = share_lo(ns) + (threadIdx.x >> 5), sl##_end = share_hi(ns); sl < sl##_end; \
       sl += (blockDim.x >> 5))

// Per-thread partial sums of the block, [2 MT][threads] doubles of dynamic
// shared memory (16 KB for one column, 64 KB for four).
extern __shared__ double g_part[];

// partial sums red[slot][c][block] -> dst[c] (shared) in every block, and
// with dst2 also red[slot2][c][block] -> dst2[c]; warp v sums value v, so the
// values are reduced on different SM sub-partitions
template <int MT>
__device__ __forceinline__ void reduce_slot(const double* red, int slot, int m, double* dst, int slot2 = 0,
                                            double* dst2 = nullptr) {
  const int G = gridDim.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = dst2 ? 2 * m : m;
  if (w < nv) {
    const int c = w < m ? w : w - m;
    const double* p = red + (size_t(w < m ? slot : slot2) * MT + c) * G;
    double t = 0.0;
    for (int b = lane; b < G; b += 32) t += p[b];
    t = warp_sum(t);
    if (lane == 0) (w < m ? dst : dst2)[c] = t;
  }
  __syncthreads();
}

// Block sums of acc[c], c < m, written to red[slot][c][blockIdx] (and of
// acc2[c] to red[slot2][c][blockIdx]).  Every thread stores its partials;
// then wpc warps per value (4 for one or two values, 2 for up to four, else
// 1) each add a contiguous share with all 32 lanes busy and finish with one
// shuffle tree.  Consecutive warps sit on different SM sub-partitions, so the
// FP64 adds of the values proceed in parallel instead of queueing behind one
// warp.  Fixed order: deterministic.
template <int MT, typename T>
__device__ __forceinline__ void write_partials(double* red, int slot, int m, const T* acc, Sh<MT>& s,
                                               const T* acc2 = nullptr, int slot2 = 0) {
  constexpr int NT = threads_for<MT>();
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int nv = acc2 ? 2 * m : m;
#pragma unroll
  for (int c = 0; c < MT; ++c)
    if (c < m) {
      g_part[c * NT + tid] = (double)acc[c];
      if (acc2) g_part[(m + c) * NT + tid] = (double)acc2[c];
    }
  __syncthreads();
  const int wpc = (nv <= 2) ? 4 : (nv <= 4 ? 2 : 1);
  const int span = NT / wpc;
  if (w < nv * wpc) {
    const int v = w / wpc, q = w - v * wpc;
    const double* p = g_part + v * NT + q * span;
    double t = 0.0;
    for (int i = lane; i < span; i += 32) t += p[i];
    t = warp_sum(t);
    if (lane == 0) s.quart[v * 4 + q] = t;
  }
  __syncthreads();
  if (tid < nv) {
    double t = s.quart[tid * 4];
    for (int q = 1; q < wpc; ++q) t += s.quart[tid * 4 + q];
    const int c = tid < m ? tid : tid - m;
    red[(size_t(tid < m ? slot : slot2) * MT + c) * gridDim.x + blockIdx.x] = t;
  }
}

// Vector layouts: the caller's b and x are column-major (element (i, c) at
// i + c ld); the solver's own vectors r, p, q, z (and the inner ones) are
// interleaved, element (i, c) at i MT + c, so the gather of X(j, :) in the
// SpMV is one contiguous MT-value load instead of MT scattered ones.
template <int MT>
__device__ __forceinline__ int64_t wix(int64_t i, int c) {
  return i * MT + c;
}

// The MT values X(j, 0..MT-1) of an interleaved vector (16-byte loads).
template <int MT, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ X, int64_t j, T* v) {
  if constexpr (MT == 1) {
    v[0] = X[j];
  } else if constexpr (sizeof(T) == 8) {
    const double2* q = reinterpret_cast<const double2*>(X + j * MT);
#pragma unroll
    for (int h = 0; h < MT / 2; ++h) {
      const double2 t = q[h];
      v[2 * h] = t.x;
      v[2 * h + 1] = t.y;
    }
  } else {
    const float4* q = reinterpret_cast<const float4*>(X + j * MT);
#pragma unroll
    for (int h = 0; h < MT / 4; ++h) {
      const float4 t = q[h];
      v[4 * h] = t.x;
      v[4 * h + 1] = t.y;
      v[4 * h + 2] = t.z;
      v[4 * h + 3] = t.w;
    }
  }
}

// Y(:,c) = A X(:,c) for columns with mask[c] (SELL-32, one row per lane);
// optionally dacc[c] += W(row,c) * Y(row,c) (and dacc2[c] += W(row,c)^2).
// Y and W are interleaved; X is
// interleaved (XI) or the caller's column-major x (stride ld).  The entry
// loop is unrolled by 4 so the loads of four entries are in flight before
// their gathers.
template <int MT, typename T, bool XI>
__device__ __forceinline__ void spmv_cols(const Sell& A, const T* __restrict__ X, int64_t ld, T* __restrict__ Y,
                                          int m, const int* mask, const T* __restrict__ W, T* dacc,
                                          T* dacc2 = nullptr) {
  const T* __restrict__ vals = (sizeof(T) == 8) ? (const T*)A.val : (const T*)A.val32;
  const int lane = threadIdx.x & 31;
  int msk[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) msk[c] = (c < m) && mask[c];
  auto gather = [&](int64_t jj, T* xv) {
    if constexpr (XI) {
      load_row<MT, T>(X, jj, xv);
    } else {
#pragma unroll
      for (int c = 0; c < MT; ++c) xv[c] = msk[c] ? X[jj + c * ld] : T(0);
    }
  };
  FOR_BLOCK_SLICES(sl, A.nslices) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    T acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    int32_t k = 0;
    constexpr int U = (MT == 1) ? 4 : 2;  // entries in flight (register budget)
    for (; k + U <= len; k += U) {
      T a[U];
      int64_t j[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = vals[base + (k + u) * 32];
        j[u] = A.col[base + (k + u) * 32];
      }
      T xv[U][MT];
#pragma unroll
      for (int u = 0; u < U; ++u) gather(j[u], xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < MT; ++c)
          if (msk[c]) acc[c] = fma(a[u], xv[u][c], acc[c]);
    }
    for (; k < len; ++k) {
      const T av = vals[base + k * 32];
      const int64_t jj = A.col[base + k * 32];
      T xv[MT];
      gather(jj, xv);
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) acc[c] = fma(av, xv[c], acc[c]);
    }
    if (row >= 0) {
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) {
          Y[wix<MT>(row, c)] = acc[c];
          if (W) {
            const T wv = W[wix<MT>(row, c)];
            dacc[c] = fma(wv, acc[c], dacc[c]);
            if (dacc2) dacc2[c] = fma(wv, wv, dacc2[c]);
          }
        }
    }
  }
}

template <int MT, typename T>
__device__ bool inner_cg(const SolverArgs& a, Sh<MT>& s) {
  // z = M^{-1} r for active columns, CG to relative residual itol (zero start).
  T* const r = (T*)a.r;
  T* const z = (T*)a.z;
  T* const ir = (T*)a.ir;
  T* const ip = (T*)a.ip;
  T* const iq = (T*)a.iq;
  const int m = a.m;
  const int64_t n = a.n;
  T acc[MT];
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    s.iact[c] = s.act[c] && s.rr[c] > 0.0;
    s.irr[c] = s.rr[c];
    s.irn0[c] = sqrt(s.rr[c]);
    s.iit[c] = 0;
  }
  __syncthreads();
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
      if (s.act[c]) {
        const T rv = r[wix<MT>(i, c)];
        z[wix<MT>(i, c)] = T(0);
        ir[wix<MT>(i, c)] = rv;
        ip[wix<MT>(i, c)] = rv;
      }
  if (!grid_sync(a.bar)) return false;
  for (int j = 1; j <= a.imaxit; ++j) {
    int any = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) any |= s.iact[c];
    if (!any) break;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T, true>(a.M, ip, 0, iq, m, s.iact, ip, acc);
    write_partials<MT, T>(a.red, 2, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 2, m, s.val);
    if (threadIdx.x < m) s.ia[threadIdx.x] = s.iact[threadIdx.x] ? s.irr[threadIdx.x] / s.val[threadIdx.x] : 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.iact[c]) {
          const int64_t o = wix<MT>(i, c);
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
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.iact[c]) {
          const int64_t o = wix<MT>(i, c);
          ip[o] = fma((T)s.ia[c], ip[o], ir[o]);
        }
    if (!grid_sync(a.bar)) return false;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long t = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) t += s.iit[c];
    *a.in_out += t;
  }
  return true;
}

// ---- mode 3: the V-cycle preconditioner z = V(r), FP32 work
//
// Section 2.3's representation A^{-1} = U B^{-1} U^T + Psi (Psi^T A Psi)^{-1}
// Psi^T (and its K-level form) applied as a symmetric V-cycle over the
// decomposition's levels: on level k a Chebyshev smoother of D^{-1} A^(k)
// (the fine-scale part; interval [hi / 30, hi], hi the Gershgorin bound),
// restriction by Psi^(k+1)^T, the same cycle on level k + 1, prolongation by
// Psi^(k+1), the same smoother again; the coarsest level by its dense
// inverse.  Every step is one pass over a level's rows followed by a grid
// barrier; vectors are MT-interleaved FP32, the outer iteration stays FP64.

// per_row(row, acc) for every row of the SELL matrix A, acc = A(row, :) X
template <int MT, typename F>
__device__ __forceinline__ void mg_rows(const Sell& A, const float* __restrict__ X, F&& per_row) {
  const int lane = threadIdx.x & 31;
  FOR_BLOCK_SLICES(sl, A.nslices) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    float acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.f;
    int32_t k = 0;
    for (; k + 2 <= len; k += 2) {
      const float a0 = A.val32[base + k * 32], a1 = A.val32[base + (k + 1) * 32];
      const int64_t j0 = A.col[base + k * 32], j1 = A.col[base + (k + 1) * 32];
      float x0[MT], x1[MT];
      load_row<MT, float>(X, j0, x0);
      load_row<MT, float>(X, j1, x1);
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = fmaf(a1, x1[c], fmaf(a0, x0[c], acc[c]));
    }
    if (k < len) {
      const float a0 = A.val32[base + k * 32];
      const int64_t j0 = A.col[base + k * 32];
      float x0[MT];
      load_row<MT, float>(X, j0, x0);
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = fmaf(a0, x0[c], acc[c]);
    }
    if (row >= 0) per_row(row, acc);
  }
}

// The same for a CSR matrix with g lanes per row (long rows of the coarse
// Galerkin matrices and of Psi^T): the group's lanes load consecutive
// entries, then add their partial sums by shuffles; the group's first lane
// calls per_row.  Rows are split into one contiguous share per block.
template <int MT, int G, typename F>
__device__ __forceinline__ void mg_rows_csr_g(const Csr32& A, const float* __restrict__ X, F&& per_row) {
  const int sub = threadIdx.x & (G - 1);
  const int64_t lo = share_lo(A.nrows), hi = share_hi(A.nrows);
  const int ngrp = blockDim.x / G;
  // every lane of a group runs the same number of rounds (the shuffles need the whole group)
  for (int64_t r0 = lo; r0 < hi; r0 += ngrp) {
    const int64_t row = r0 + threadIdx.x / G;
    float acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.f;
    if (row < hi) {
      const int32_t e0 = A.rowptr[row], e1 = A.rowptr[row + 1];
      for (int32_t e = e0 + sub; e < e1; e += G) {
        const float a = A.val[e];
        float xv[MT];
        load_row<MT, float>(X, A.col[e], xv);
#pragma unroll
        for (int c = 0; c < MT; ++c) acc[c] = fmaf(a, xv[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < MT; ++c)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
    if (row < hi && sub == 0) per_row((int32_t)row, acc);
  }
}

// per_row over a V-cycle matrix: CSR with g lanes per row when its rows are
// long, else the SELL copy with one row per lane
template <int MT, typename F>
__device__ __forceinline__ void mg_apply(const Sell& S, const Csr32& C, const float* __restrict__ X, F&& per_row) {
  if (C.g == 32)
    mg_rows_csr_g<MT, 32>(C, X, per_row);
  else if (C.g == 8)
    mg_rows_csr_g<MT, 8>(C, X, per_row);
  else
    mg_rows<MT>(S, X, per_row);
}

// The buffer holding level k's iterate after its pre-smoothing (deg - 1
// ping-pong swaps) and after its post-smoothing (deg more).
__device__ __forceinline__ float* mg_xpre(const MGLevel& L, int deg) { return ((deg - 1) & 1) ? L.x2 : L.x; }
__device__ __forceinline__ float* mg_xpost(const MGLevel& L, int deg) {
  return ((2 * deg - 1) & 1) ? L.x2 : L.x;
}

// z = V(r) for the columns with act[c] (r, z: the outer solver's FP64
// interleaved vectors); the other columns' z is left alone.
template <int MT>
__device__ __forceinline__ bool mg_vcycle(const SolverArgs& a, const int* act) {
  const double* __restrict__ r0 = (const double*)a.r;
  double* __restrict__ z0 = (double*)a.z;
  const int K = a.mg_K, deg = a.mg_deg;
  int on[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) on[c] = (c < a.m) && act[c];
  // ---- down: pre-smoothing from x = 0, residual, restriction
  for (int k = 0; k < K; ++k) {
    const MGLevel& L = a.mg[k];
    float* x = L.x;
    float* x2 = L.x2;
    float* __restrict__ rr = L.r;
    float* __restrict__ dd = L.d;
    const float* __restrict__ dinv = L.dinv;
    const float c0 = L.c2[0];
    FOR_BLOCK_SHARE(i, L.n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) {
        const int64_t o = wix<MT>(i, c);
        float rv;
        if (k == 0) {
          rv = on[c] ? (float)r0[o] : 0.f;
          rr[o] = rv;
        } else {
          rv = rr[o];
        }
        const float dv = c0 * dinv[i] * rv;
        dd[o] = dv;
        x[o] = dv;
      }
    if (!grid_sync(a.bar)) return false;
    for (int st = 1; st < deg; ++st) {
      const float c1 = L.c1[st], c2 = L.c2[st];
      const float* xs = x;
      float* xd = x2;
      mg_apply<MT>(L.A, L.cA, xs, [&](int32_t row, const float* acc) {
#pragma unroll
        for (int c = 0; c < MT; ++c) {
          const int64_t o = wix<MT>(row, c);
          const float dv = fmaf(c1, dd[o], c2 * dinv[row] * (rr[o] - acc[c]));
          dd[o] = dv;
          xd[o] = xs[o] + dv;
        }
      });
      if (!grid_sync(a.bar)) return false;
      float* t = x;
      x = x2;
      x2 = t;
    }
    // residual of the pre-smoothed iterate (into d), then its restriction
    {
      const float* xs = x;
      mg_apply<MT>(L.A, L.cA, xs, [&](int32_t row, const float* acc) {
#pragma unroll
        for (int c = 0; c < MT; ++c) {
          const int64_t o = wix<MT>(row, c);
          dd[o] = rr[o] - acc[c];
        }
      });
    }
    if (!grid_sync(a.bar)) return false;
    float* __restrict__ rnext = (k + 1 < K) ? a.mg[k + 1].r : a.mg_rK;
    mg_apply<MT>(L.PT, L.cPT, dd, [&](int32_t row, const float* acc) {
#pragma unroll
      for (int c = 0; c < MT; ++c) rnext[wix<MT>(row, c)] = acc[c];
    });
    if (!grid_sync(a.bar)) return false;
  }
  // ---- coarsest: x_K = A_K^{-1} r_K (symmetric inverse, row i read as column i), one warp per row
  {
    const int64_t nK = a.mg_nK;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t row = warp; row < nK; row += nw) {
      float acc[MT];
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = 0.f;
      for (int64_t j = lane; j < nK; j += 32) {
        const float kv = a.mg_kinv[j + row * nK];
        float xv[MT];
        load_row<MT, float>(a.mg_rK, j, xv);
#pragma unroll
        for (int c = 0; c < MT; ++c) acc[c] = fmaf(kv, xv[c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < MT; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0) a.mg_xK[wix<MT>(row, c)] = acc[c];
      }
    }
    if (!grid_sync(a.bar)) return false;
  }
  // ---- up: prolongation, post-smoothing
  for (int k = K - 1; k >= 0; --k) {
    const MGLevel& L = a.mg[k];
    float* x = mg_xpre(L, deg);
    float* x2 = (x == L.x) ? L.x2 : L.x;
    float* __restrict__ rr = L.r;
    float* __restrict__ dd = L.d;
    const float* __restrict__ dinv = L.dinv;
    const float* __restrict__ xc = (k + 1 < K) ? mg_xpost(a.mg[k + 1], deg) : a.mg_xK;
    {
      float* xw = x;
      mg_apply<MT>(L.P, L.cP, xc, [&](int32_t row, const float* acc) {
#pragma unroll
        for (int c = 0; c < MT; ++c) xw[wix<MT>(row, c)] += acc[c];
      });
    }
    if (!grid_sync(a.bar)) return false;
    for (int st = 0; st < deg; ++st) {
      const float c1 = L.c1[st], c2 = L.c2[st];
      const bool out = (k == 0) && (st == deg - 1);
      const float* xs = x;
      float* xd = x2;
      mg_apply<MT>(L.A, L.cA, xs, [&](int32_t row, const float* acc) {
#pragma unroll
        for (int c = 0; c < MT; ++c) {
          const int64_t o = wix<MT>(row, c);
          const float g = c2 * dinv[row] * (rr[o] - acc[c]);
          const float dv = (st == 0) ? g : fmaf(c1, dd[o], g);
          dd[o] = dv;
          const float xn = xs[o] + dv;
          xd[o] = xn;
          if (out && on[c]) z0[o] = (double)xn;
        }
      });
      if (!grid_sync(a.bar)) return false;
      float* t = x;
      x = x2;
      x2 = t;
    }
  }
  return true;
}

// z = p(D^{-1} A) D^{-1} r for the columns with act[c] (mode 4): deg steps
// of the Chebyshev iteration for A z = r from z = 0, FP32, one pass over the
// rows and one grid barrier per step and no reduction, so a preconditioned
// iteration trades deg - 1 cheap FP32 SpMVs for the grid-wide reduction
// rounds (and FP64 SpMVs) of the CG iterations it saves.  The other columns'
// z is left alone.
template <int MT>
__device__ __forceinline__ bool cheb_prec(const SolverArgs& a, const int* act) {
  const PolyPrec& P = a.poly;
  const double* __restrict__ r0 = (const double*)a.r;
  double* __restrict__ z0 = (double*)a.z;
  const int deg = P.deg;
  int on[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) on[c] = (c < a.m) && act[c];
  float* x = P.x;
  float* x2 = P.x2;
  float* __restrict__ rr = P.r;
  float* __restrict__ dd = P.d;
  const float* __restrict__ dinv = P.dinv;
  const float c0 = P.c2[0];
  FOR_BLOCK_SHARE(i, a.n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) {
      const int64_t o = wix<MT>(i, c);
      const float rv = on[c] ? (float)r0[o] : 0.f;
      rr[o] = rv;
      const float dv = c0 * dinv[i] * rv;
      dd[o] = dv;
      x[o] = dv;
      if (deg == 1 && on[c]) z0[o] = (double)dv;
    }
  if (!grid_sync(a.bar)) return false;
  for (int st = 1; st < deg; ++st) {
    const float c1 = P.c1[st], c2 = P.c2[st];
    const bool out = (st == deg - 1);
    const float* xs = x;
    float* xd = x2;
    mg_apply<MT>(a.A, P.cA, xs, [&](int32_t row, const float* acc) {
#pragma unroll
      for (int c = 0; c < MT; ++c) {
        const int64_t o = wix<MT>(row, c);
        const float dv = fmaf(c1, dd[o], c2 * dinv[row] * (rr[o] - acc[c]));
        dd[o] = dv;
        const float xn = xs[o] + dv;
        xd[o] = xn;
        if (out && on[c]) z0[o] = (double)xn;
      }
    });
    if (!grid_sync(a.bar)) return false;
    float* t = x;
    x = x2;
    x2 = t;
  }
  return true;
}

// Mode 0: CG in the Chronopoulos-Gear form: r^T r and r^T A r are both
// formed in the SpMV pass (w = A r), so an iteration has one reduction round
// (block sums, grid barrier, partials) and one plain grid barrier before the
// next SpMV; same iterates as Hestenes-Stiefel CG in exact arithmetic.  The
// convergence test sees r^T r of the last update in the next pass, so a
// converged column has done one SpMV more than it needed.
// On entry r = b - A x0 is complete and s.rr = r^T r, s.act, s.bn are set.
template <int MT, typename T>
__device__ bool cgcg(const SolverArgs& a, Sh<MT>& s) {
  T* const r = (T*)a.r;
  T* const p = (T*)a.p;
  T* const x = (T*)a.x;
  T* const w = (T*)a.z;
  T* const sv = (T*)a.q;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  T acc[MT], acc2[MT];
  for (int it = 1;; ++it) {
    int any = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) any |= s.act[c];
    if (!any) break;
    // w = A r; delta = r^T w, gamma = r^T r
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = T(0);
    spmv_cols<MT, T, true>(a.A, r, 0, w, m, s.act, r, acc, acc2);
    write_partials<MT, T>(a.red, 0, m, acc, s, acc2, 1);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 0, m, s.val, 1, s.val2);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        const double g = s.val2[c], dl = s.val[c];
        if (it > 1 && g <= a.tol * a.tol * s.bn[c] * s.bn[c]) {
          s.act[c] = 0;  // converged after update it - 1
        } else if (it <= a.maxit) {
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
          s.it[c] = it;
        }
      }
    }
    __syncthreads();
    if (it > a.maxit) break;  // columns still active report no convergence
    // p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s
    const bool first = (it == 1);
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.act[c]) {
          const int64_t o = wix<MT>(i, c), ox = i + c * ld;
          const T be = (T)s.val2[c], al = (T)s.alpha[c];
          const T rv0 = r[o];
          const T pv = first ? rv0 : fma(be, p[o], rv0);
          const T svv = first ? w[o] : fma(be, sv[o], w[o]);
          p[o] = pv;
          sv[o] = svv;
          x[ox] = fma(al, pv, x[ox]);
          r[o] = fma(-al, svv, rv0);
        }
    if (!grid_sync(a.bar)) return false;
  }
  return true;
}

// FP64 residual of the reliable update: rr32 = (float)(b64 - A x64), partial
// sums of its square; FP64 SELL SpMV (matrix values in FP64).
template <int MT, typename T>
__device__ void reliable_residual(const SolverArgs& a, const int* mask, T* r32, double* acc) {
  const Sell& A = a.A;
  const int m = a.m;
  const int64_t ld = a.ld;
  const int lane = threadIdx.x & 31;
  FOR_BLOCK_SLICES(sl, A.nslices) {
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
          r32[wix<MT>(row, c)] = (T)rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    }
  }
}

// Mode 0 with residual replacement (reliable updates; van der Vorst and Ye
// 2000, as used for mixed-precision CG): Hestenes-Stiefel CG whose
// recurrences run in T (FP32 in the mixed mode) while x accumulates in FP64.
// Whenever the recurrence residual has dropped 100x since the last
// replacement -- and before convergence is accepted -- r is replaced by the
// FP64 residual b - A x.  The Krylov recurrence is kept (no restart);
// alpha = r^T r / p^T A p is computed directly, so a replacement needs no
// further correction.  A column stops unconverged (conv = 0) when its true
// residual stalls across a replacement or p^T A p <= 0 in FP32 -- FP32
// cannot resolve directions whose Rayleigh quotient is below about
// u_32 ||A||, as for the 1e-6-shifted Laplacians -- and the caller finishes
// it with FP64 CG from the current x.
template <int MT, typename T>
__device__ bool cg_rel(const SolverArgs& a, Sh<MT>& s) {
  T* const r = (T*)a.r;
  T* const p = (T*)a.p;
  T* const q = (T*)a.q;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  T acc[MT];
  double dacc[MT];
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) {
    all1[c] = 1;
    dacc[c] = 0.0;
  }
  if (!a.x0)
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) a.x64[i + c * ld] = 0.0;
  if (!grid_sync(a.bar)) return false;
  reliable_residual<MT, T>(a, all1, r, dacc);
  write_partials<MT, double>(a.red, 1, m, dacc, s);
#pragma unroll
  for (int c = 0; c < MT; ++c) dacc[c] = 0.0;
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) dacc[c] = fma(a.b64[i + c * ld], a.b64[i + c * ld], dacc[c]);
  write_partials<MT, double>(a.red, 0, m, dacc, s);
  if (!grid_sync(a.bar)) return false;
  reduce_slot<MT>(a.red, 0, m, s.bn);
  reduce_slot<MT>(a.red, 1, m, s.rr);
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    s.bn[c] = sqrt(s.bn[c]);
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.rr[c]) <= a.tol * s.bn[c]);
    s.ok[c] = !s.act[c];
    s.it[c] = 0;
    s.irn0[c] = sqrt(s.rr[c]);  // residual norm at the last replacement
    s.due[c] = 0;
    s.stag[c] = 0;
  }
  __syncthreads();
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
      if (s.act[c]) p[wix<MT>(i, c)] = r[wix<MT>(i, c)];
  if (!grid_sync(a.bar)) return false;
  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) any |= s.act[c];
    if (!any) break;
    // q = A p, p^T q
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T, true>(a.A, p, 0, q, m, s.act, p, acc);
    write_partials<MT, T>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 0, m, s.val);
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        if (!(s.val[c] > 0.0)) {
          // FP32 cannot resolve A below u_32 ||A||: the column stops
          // unconverged (the caller finishes it in FP64); in FP64 it is an error
          s.act[c] = 0;
          if (sizeof(T) == 8 && blockIdx.x == 0) atomicExch(a.bar.status, (int)DEV_NOTSPD);
        } else {
          s.alpha[c] = s.rr[c] / s.val[c];
        }
      }
    }
    __syncthreads();
    // x += alpha p (FP64), r -= alpha q, r^T r
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.act[c]) {
          const int64_t o = wix<MT>(i, c), ox = i + c * ld;
          const T al = (T)s.alpha[c];
          a.x64[ox] = fma(s.alpha[c], (double)p[o], a.x64[ox]);
          const T rv = fma(-al, q[o], r[o]);
          r[o] = rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    write_partials<MT, T>(a.red, 1, m, acc, s);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 1, m, s.val2);
    // the recurrence drifts from the true residual: replace it after every
    // two decades of reduction and before accepting convergence
    int need = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
      if (s.act[c] && (sqrt(s.val2[c]) <= 0.01 * s.irn0[c] || sqrt(s.val2[c]) <= a.tol * s.bn[c])) need = 1;
    if (need) {
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        s.due[c] = s.act[c] && sqrt(s.val2[c]) <= 0.01 * s.irn0[c];
      }
      int msk[MT];
#pragma unroll
      for (int c = 0; c < MT; ++c) {
        msk[c] = (c < m) && s.act[c];
        dacc[c] = 0.0;
      }
      reliable_residual<MT, T>(a, msk, r, dacc);  // x64 complete: barrier above
      write_partials<MT, double>(a.red, 2, m, dacc, s);
      if (!grid_sync(a.bar)) return false;
      reduce_slot<MT>(a.red, 2, m, s.val2);  // true residuals replace the recurrence ones
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c]) {
          // two decades of recurrence reduction that left the true residual
          // above half its last value: stalled
          const double tn = sqrt(s.val2[c]);
          s.stag[c] = s.due[c] && tn > 0.5 * s.irn0[c];
          s.irn0[c] = tn;
        }
      }
    }
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (s.act[c]) {
        s.it[c] = it;
        const double gn = s.val2[c];
        s.val[c] = gn / s.rr[c];  // beta
        s.rr[c] = gn;
        // convergence is accepted on a replaced (true) residual only
        if (need && sqrt(gn) <= a.tol * s.bn[c]) {
          s.act[c] = 0;
          s.ok[c] = 1;
        } else if (need && s.stag[c]) {
          s.act[c] = 0;  // stalled above tol: reported unconverged
        }
      }
    }
    __syncthreads();
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.act[c]) {
          const int64_t o = wix<MT>(i, c);
          p[o] = fma((T)s.val[c], p[o], r[o]);
        }
    if (!grid_sync(a.bar)) return false;
  }
  return true;
}

// ---- double-float arithmetic (the level-0 CG of MMD_MIXED)
//
// A value is the unevaluated sum hi + lo of two FP32 numbers, |lo| <= half
// an ulp of hi: about 48 significant bits, the exponent range of FP32.  The
// error-free transformations are Knuth's two-sum (s + e = a + b exactly) and
// the FMA two-product (p + e = a b exactly); the pair operations follow
// Dekker (1971) and the GPU formulation of Thall (2006), "sloppy" addition
// (the low parts added without their own two-sum: error below 2^-44 of the
// operands' magnitude).  Every step uses the rounded intrinsics, so the
// compiler neither contracts a step into an FMA nor reassociates.  GB300
// issues FP32 about seventy times faster than FP64 (one FP64 FMA per 64
// cycles per warp on an SM sub-partition), so the 15 FP32 operations of a
// pair FMA cost about a quarter of one FP64 FMA.
struct dd {
  float hi, lo;
};
__device__ __forceinline__ dd dd_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dd_val(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dd dd_renorm(float s, float e) {  // |s| >= |e| or s = 0
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return dd_renorm(s, e);
}
// a b + c
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  return dd_renorm(s, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_warp_sum(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd t;
    t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, t);
  }
  return v;
}

// The MT values X(j, 0..MT-1) of an interleaved pair vector.
template <int MT>
__device__ __forceinline__ void load_row_dd(const dd* __restrict__ X, int64_t j, dd* v) {
  if constexpr (MT == 1) {
    const float2 t = reinterpret_cast<const float2*>(X)[j];
    v[0] = {t.x, t.y};
  } else {
    const float4* q = reinterpret_cast<const float4*>(X + j * MT);
#pragma unroll
    for (int h = 0; h < MT / 2; ++h) {
      const float4 t = q[h];
      v[2 * h] = {t.x, t.y};
      v[2 * h + 1] = {t.z, t.w};
    }
  }
}

// Y(:,c) = A X(:,c) in pair arithmetic (SELL-32, one row per lane, values
// val2), and dacc[c] += W(row,c) Y(row,c), dacc2[c] += W(row,c)^2.
template <int MT>
__device__ __forceinline__ void spmv_dd(const Sell& A, const dd* __restrict__ X, dd* __restrict__ Y, int m,
                                        const int* mask, const dd* __restrict__ W, dd* dacc, dd* dacc2) {
  const float2* __restrict__ vals = A.val2;
  const int lane = threadIdx.x & 31;
  int msk[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) msk[c] = (c < m) && mask[c];
  FOR_BLOCK_SLICES(sl, A.nslices) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    dd acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = {0.f, 0.f};
    int32_t k = 0;
    constexpr int U = (MT == 1) ? 4 : 2;  // entries in flight
    for (; k + U <= len; k += U) {
      float2 a[U];
      int64_t j[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = vals[base + (k + u) * 32];
        j[u] = A.col[base + (k + u) * 32];
      }
      dd xv[U][MT];
#pragma unroll
      for (int u = 0; u < U; ++u) load_row_dd<MT>(X, j[u], xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < MT; ++c)
          if (msk[c]) acc[c] = dd_fma({a[u].x, a[u].y}, xv[u][c], acc[c]);
    }
    for (; k < len; ++k) {
      const float2 av = vals[base + k * 32];
      dd xv[MT];
      load_row_dd<MT>(X, A.col[base + k * 32], xv);
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) acc[c] = dd_fma({av.x, av.y}, xv[c], acc[c]);
    }
    if (row >= 0) {
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (msk[c]) {
          Y[wix<MT>(row, c)] = acc[c];
          const dd wv = W[wix<MT>(row, c)];
          dacc[c] = dd_fma(wv, acc[c], dacc[c]);
          dacc2[c] = dd_fma(wv, wv, dacc2[c]);
        }
    }
  }
}

// Block sums of acc[c] (slot) and acc2[c] (slot2), c < m, in pair
// arithmetic: warp shuffles, one pair per warp in shared memory, then warp v
// adds the block's warp pairs of value v and stores red[slot][c][blockIdx]
// as a float2; no FP64 instruction.  Fixed order: deterministic.
template <int MT>
__device__ __forceinline__ void write_partials_dd(float2* red, int slot, int m, const dd* acc, int slot2,
                                                  const dd* acc2) {
  float2* sh = reinterpret_cast<float2*>(g_part);  // [2 MT][32]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < MT; ++c)
    if (c < m) {
      const dd a = dd_warp_sum(acc[c]);
      const dd b = dd_warp_sum(acc2[c]);
      if (lane == 0) {
        sh[c * 32 + w] = make_float2(a.hi, a.lo);
        sh[(MT + c) * 32 + w] = make_float2(b.hi, b.lo);
      }
    }
  __syncthreads();
  if (w < 2 * m) {
    const int v = w < m ? w : MT + (w - m);
    const int c = w < m ? w : w - m;
    dd t = {0.f, 0.f};
    if (lane < nw) {
      const float2 q = sh[v * 32 + lane];
      t = {q.x, q.y};
    }
    t = dd_warp_sum(t);
    if (lane == 0) red[(size_t(w < m ? slot : slot2) * MT + c) * gridDim.x + blockIdx.x] = make_float2(t.hi, t.lo);
  }
}

// red[slot][c][*] -> dst[c] and red[slot2][c][*] -> dst2[c] (FP64, shared),
// the partials added in pair arithmetic.
template <int MT>
__device__ __forceinline__ void reduce_slot_dd(const float2* red, int slot, int m, double* dst, int slot2,
                                               double* dst2) {
  const int G = gridDim.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 2 * m) {
    const int c = w < m ? w : w - m;
    const float2* p = red + (size_t(w < m ? slot : slot2) * MT + c) * G;
    dd t = {0.f, 0.f};
    for (int b = lane; b < G; b += 32) t = dd_add(t, {p[b].x, p[b].y});
    t = dd_warp_sum(t);
    if (lane == 0) (w < m ? dst : dst2)[c] = dd_val(t);
  }
  __syncthreads();
}

// r = b - A x in FP64 (x: the caller's FP64 column-major solution; q64:
// interleaved FP64 scratch), stored as pairs in r and rr[c] = ||r_c||^2;
// columns without mask[c] are skipped.  With first, x = 0 is taken and no
// product is formed.
template <int MT>
__device__ bool dd_true_residual(const SolverArgs& a, Sh<MT>& s, const int* mask, bool first, double* rr) {
  const double* __restrict__ b = (const double*)a.b;
  const double* __restrict__ x = (const double*)a.x;
  double* q64 = (double*)a.ip;
  dd* r = (dd*)a.r;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  double dummy[MT];
  if (!first) {
    spmv_cols<MT, double, false>(a.A, x, ld, q64, m, mask, nullptr, dummy);
    if (!grid_sync(a.bar)) return false;
  }
  double acc[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) acc[c] = 0.0;
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m && mask[c]) {
      const int64_t o = wix<MT>(i, c);
      const double rv = first ? b[i + c * ld] : b[i + c * ld] - q64[o];
      r[o] = dd_of(rv);
      acc[c] = fma(rv, rv, acc[c]);
    }
  write_partials<MT, double>(a.red, 3, m, acc, s);
  if (!grid_sync(a.bar)) return false;
  reduce_slot<MT>(a.red, 3, m, rr);
  return true;
}

// Mode 0 in double-float (MMD_MIXED at level 0): the Chronopoulos-Gear CG of
// cgcg with r, p, s = A p, w = A r and the iterate held as FP32 pairs and
// the matrix as its pair copy; the scalars alpha, beta stay FP64.  When the
// recurrence residual meets tol, x (FP64) is formed and its FP64 residual
// b - A x is checked; a column above tol restarts CG from its current x with
// that residual (at most three restarts, and only while the true residual
// falls), else it stops unconverged (conv = 0) and the caller finishes it
// in FP64.  On exit x holds the solution in FP64.
template <int MT>
__global__ void __launch_bounds__(threads_for<MT>(), 1) dd_cg_kernel(SolverArgs a) {
  __shared__ Sh<MT> s;
  __shared__ float2 s_ab[2 * MT];  // alpha, beta of the columns as pairs
  __shared__ double s_true[MT], s_last[MT];
  __shared__ long long s_base[MT];
  grid_sync_init();
  const double* __restrict__ b = (const double*)a.b;
  double* __restrict__ x = (double*)a.x;
  dd* const r = (dd*)a.r;
  dd* const p = (dd*)a.p;
  dd* const sv = (dd*)a.q;
  dd* const w = (dd*)a.z;
  dd* const xd = (dd*)a.ir;
  float2* const red2 = (float2*)a.red;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) all1[c] = 1;
  // iterate as pairs; ||b||
  double acc[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) acc[c] = 0.0;
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) {
      const int64_t o = wix<MT>(i, c), ox = i + c * ld;
      if (a.x0) {
        xd[o] = dd_of(x[ox]);
      } else {
        xd[o] = {0.f, 0.f};
        x[ox] = 0.0;
      }
      acc[c] = fma(b[ox], b[ox], acc[c]);
    }
  write_partials<MT, double>(a.red, 2, m, acc, s);
  if (!grid_sync(a.bar)) return;
  reduce_slot<MT>(a.red, 2, m, s.bn);
  if (!dd_true_residual<MT>(a, s, all1, !a.x0, s_true)) return;
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    s.bn[c] = sqrt(s.bn[c]);
    s.rr[c] = s_true[c];
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.rr[c]) <= a.tol * s.bn[c]);
    s.ok[c] = !s.act[c];
    s.it[c] = 0;
    s_last[c] = sqrt(s.rr[c]);
  }
  __syncthreads();
  for (int pass = 0;; ++pass) {
    if (threadIdx.x < m) s_base[threadIdx.x] = s.it[threadIdx.x];
    __syncthreads();
    for (int it = 1;; ++it) {
      int run[MT], any = 0;
#pragma unroll
      for (int c = 0; c < MT; ++c) {
        run[c] = (c < m) && s.act[c] == 1;
        any |= run[c];
      }
      if (!any) break;
      // w = A r; delta = r^T w, gamma = r^T r
      dd pa[MT], pb[MT];
#pragma unroll
      for (int c = 0; c < MT; ++c) pa[c] = pb[c] = {0.f, 0.f};
      spmv_dd<MT>(a.A, r, w, m, run, r, pa, pb);
      write_partials_dd<MT>(red2, 0, m, pa, 1, pb);
      if (!grid_sync(a.bar)) return;
      reduce_slot_dd<MT>(red2, 0, m, s.val, 1, s.val2);
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c] == 1) {
          const double g = s.val2[c], dl = s.val[c];
          if (it > 1 && g <= a.tol * a.tol * s.bn[c] * s.bn[c]) {
            s.act[c] = 2;  // recurrence converged after update it - 1: check the true residual
          } else if (s_base[c] + it <= a.maxit) {
            double be = 0.0, den = dl;
            if (it > 1) {
              be = g / s.rz[c];
              den = dl - be * g / s.alpha[c];
            }
            if (!(den > 0.0)) {  // not SPD at this precision: the caller finishes in FP64
              s.act[c] = 0;
            } else {
              s.rz[c] = g;
              s.alpha[c] = g / den;
              const dd al = dd_of(s.alpha[c]), bt = dd_of(be);
              s_ab[c] = make_float2(al.hi, al.lo);
              s_ab[MT + c] = make_float2(bt.hi, bt.lo);
              s.it[c] = s_base[c] + it;
            }
          } else {
            s.act[c] = 0;  // iteration cap
          }
        }
      }
      __syncthreads();
      int upd[MT];
#pragma unroll
      for (int c = 0; c < MT; ++c) upd[c] = (c < m) && s.act[c] == 1;
      const bool first = (it == 1);
      FOR_BLOCK_SHARE(i, n)
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (upd[c]) {
          const int64_t o = wix<MT>(i, c);
          const dd al = {s_ab[c].x, s_ab[c].y}, be = {s_ab[MT + c].x, s_ab[MT + c].y};
          const dd rv0 = r[o];
          const dd pv = first ? rv0 : dd_fma(be, p[o], rv0);
          const dd svv = first ? w[o] : dd_fma(be, sv[o], w[o]);
          p[o] = pv;
          sv[o] = svv;
          xd[o] = dd_fma(al, pv, xd[o]);
          r[o] = dd_fma(dd_neg(al), svv, rv0);
        }
      if (!grid_sync(a.bar)) return;
      // columns whose recurrence converged leave the loop with act = 2
      int more = 0;
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) more |= (s.act[c] == 1);
      if (!more) break;
    }
    // x = the pair iterate in FP64; true residual of the columns that converged in the recurrence
    int chk[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) chk[c] = (c < m) && s.act[c] == 2;
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) x[i + c * ld] = dd_val(xd[wix<MT>(i, c)]);
    if (!grid_sync(a.bar)) return;
    int anychk = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) anychk |= chk[c];
    if (!anychk) break;
    if (!dd_true_residual<MT>(a, s, chk, false, s_true)) return;
    if (threadIdx.x < m) {
      const int c = threadIdx.x;
      if (chk[c]) {
        const double tn = sqrt(s_true[c]);
        if (tn <= a.tol * s.bn[c]) {
          s.act[c] = 0;
          s.ok[c] = 1;
        } else if (pass < 3 && tn < 0.5 * s_last[c]) {
          s.act[c] = 1;  // restart from x with the true residual
          s.rr[c] = s_true[c];
          s_last[c] = tn;
        } else {
          s.act[c] = 0;  // stalled: reported unconverged
        }
      }
    }
    __syncthreads();
    int again = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) again |= (s.act[c] == 1);
    if (!again) break;
  }
  if (blockIdx.x == 0 && threadIdx.x < m) {
    a.it_out[threadIdx.x] = s.it[threadIdx.x];
    a.conv[threadIdx.x] = s.ok[threadIdx.x];
  }
}

// VC = 1: the instance with the V-cycle (mode 3) and polynomial (mode 4)
// preconditioners, kept apart so that the other modes' register allocation
// does not see their calls.
template <int MT, typename T, int VC>
__global__ void __launch_bounds__(threads_for<MT>(), 1) solve_kernel(SolverArgs a) {
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
  if constexpr (VC == 1 && sizeof(T) == 8) {
    if (a.mg_only) {  // one application z = V(b) or p(D^{-1}A) D^{-1} b: b and x column-major, all m columns
      FOR_BLOCK_SHARE(i, n)
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) r[wix<MT>(i, c)] = b[i + c * ld];
      if (threadIdx.x < MT) s.act[threadIdx.x] = threadIdx.x < m;
      __syncthreads();
      if (!grid_sync(a.bar)) return;
      if (!(a.mode == 4 ? cheb_prec<MT>(a, s.act) : mg_vcycle<MT>(a, s.act))) return;
      FOR_BLOCK_SHARE(i, n)
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) x[i + c * ld] = z[wix<MT>(i, c)];
      if (blockIdx.x == 0 && threadIdx.x < m) {
        a.it_out[threadIdx.x] = 1;
        a.conv[threadIdx.x] = 1;
      }
      return;
    }
  }
  if (a.mode == 0 && a.b64) {
    if (!cg_rel<MT, T>(a, s)) return;
    if (blockIdx.x == 0 && threadIdx.x < m) {
      a.it_out[threadIdx.x] = s.it[threadIdx.x];
      a.conv[threadIdx.x] = s.ok[threadIdx.x];
    }
    return;
  }
  T acc[MT], acc2[MT];
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) all1[c] = 1;
  // ---- set-up: r = b - A x0 (or b), norms
  if (a.x0) {
    spmv_cols<MT, T, false>(a.A, x, ld, q, m, all1, nullptr, nullptr);
    if (!grid_sync(a.bar)) return;
  }
#pragma unroll
  for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = T(0);
  if (a.mode == 2) {
    // r = P (b - A x0) per segment: a right-hand side projected once by the
    // caller keeps a rounding-level component along phi, as large as its
    // projected part when b was nearly parallel to phi; CG could not remove it
    FOR_BLOCK_SHARE(sg, a.nseg) {
      const int32_t s0 = a.seg_ptr[sg], s1 = a.seg_ptr[sg + 1];
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) {
        T t = T(0);
        for (int32_t i = s0; i < s1; ++i) {
          const int64_t o = i + c * ld, w = wix<MT>(i, c);
          t = fma((T)a.phi[i], a.x0 ? b[o] - q[w] : b[o], t);
        }
        for (int32_t i = s0; i < s1; ++i) {
          const int64_t o = i + c * ld, w = wix<MT>(i, c);
          const T bv = b[o];
          const T rv = fma(-(T)a.phi[i], t, a.x0 ? bv - q[w] : bv);
          if (!a.x0) x[o] = T(0);
          r[w] = rv;
          acc[c] = fma(bv, bv, acc[c]);
          acc2[c] = fma(rv, rv, acc2[c]);
        }
      }
    }
  } else {
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) {
        const int64_t o = i + c * ld, w = wix<MT>(i, c);
        const T bv = b[o];
        T rv = bv;
        if (a.x0) rv -= q[w];
        else x[o] = T(0);
        r[w] = rv;
        acc[c] = fma(bv, bv, acc[c]);
        acc2[c] = fma(rv, rv, acc2[c]);
      }
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
  FOR_BLOCK_SHARE(i, n)  // zero right-hand sides give x = 0
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
      if (s.bn[c] == 0.0) x[i + c * ld] = T(0);
  if (a.mode == 0) {
    if (!cgcg<MT, T>(a, s)) return;
    if (blockIdx.x == 0 && threadIdx.x < m) {
      a.it_out[threadIdx.x] = s.it[threadIdx.x];
      a.conv[threadIdx.x] = s.act[threadIdx.x] ? 0 : 1;
    }
    return;
  }
  T* zv = r;
  if (a.mode == 1 || a.mode == 3 || a.mode == 4) {
    if (a.mode == 1) {
      if (!inner_cg<MT, T>(a, s)) return;
    } else if constexpr (sizeof(T) == 8 && VC == 1) {
      if (a.mode == 4) {
        if (!cheb_prec<MT>(a, s.act)) return;
      } else if (!mg_vcycle<MT>(a, s.act)) {
        return;
      }
    }
    zv = z;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.act[c]) acc[c] = fma(r[wix<MT>(i, c)], z[wix<MT>(i, c)], acc[c]);
    write_partials<MT, T>(a.red, 0, m, acc, s);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 0, m, s.rz);
  } else {
    if (threadIdx.x < m) s.rz[threadIdx.x] = s.rr[threadIdx.x];
    __syncthreads();
  }
  FOR_BLOCK_SHARE(i, n)
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
      if (s.act[c]) p[wix<MT>(i, c)] = zv[wix<MT>(i, c)];
  if (!grid_sync(a.bar)) return;

  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) any |= s.act[c];
    if (!any) break;
    // q = A p, p^T q
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = T(0);
    spmv_cols<MT, T, true>(a.A, p, 0, q, m, s.act, p, acc);
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
      FOR_BLOCK_SHARE(sg, a.nseg) {
        const int32_t s0 = a.seg_ptr[sg], s1 = a.seg_ptr[sg + 1];
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m) {
          if (!s.act[c]) continue;
          const T al = (T)s.alpha[c];
          T t = T(0);
          for (int32_t i = s0; i < s1; ++i) t = fma((T)a.phi[i], q[wix<MT>(i, c)], t);
          for (int32_t i = s0; i < s1; ++i) {
            const int64_t o = wix<MT>(i, c), ox = i + c * ld;
            const T qv = fma(-(T)a.phi[i], t, q[o]);
            x[ox] = fma(al, p[o], x[ox]);
            const T rv = fma(-al, qv, r[o]);
            r[o] = rv;
            acc[c] = fma(rv, rv, acc[c]);
          }
        }
      }
    } else {
      FOR_BLOCK_SHARE(i, n)
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
          if (s.act[c]) {
            const int64_t o = wix<MT>(i, c), ox = i + c * ld;
            const T al = (T)s.alpha[c];
            x[ox] = fma(al, p[o], x[ox]);
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
    if (a.mode == 1 || a.mode == 3 || a.mode == 4) {
      // columns that just converged (-1) need no preconditioning
      if (threadIdx.x < m) {
        const int c = threadIdx.x;
        if (s.act[c] < 0) s.act[c] = 0;
        s.rr[c] = s.val2[c];
      }
      __syncthreads();
      if (a.mode == 1) {
        if (!inner_cg<MT, T>(a, s)) return;
      } else if constexpr (sizeof(T) == 8 && VC == 1) {
        if (a.mode == 4) {
          if (!cheb_prec<MT>(a, s.act)) return;
        } else if (!mg_vcycle<MT>(a, s.act)) {
          return;
        }
      }
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = T(0);
      FOR_BLOCK_SHARE(i, n)
        _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
          if (s.act[c]) {
            const int64_t o = wix<MT>(i, c);
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
    FOR_BLOCK_SHARE(i, n)
      _Pragma("unroll") for (int c = 0; c < MT; ++c) if (c < m)
        if (s.act[c]) {
          const int64_t o = wix<MT>(i, c);
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

template <int MT>
constexpr size_t dyn_smem() {
  return sizeof(double) * 2 * size_t(MT) * threads_for<MT>();
}

// the 64 KB of the four-column instance exceed the default 48 KB window
template <int MT, typename T, int VC>
void allow_smem() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(solve_kernel<MT, T, VC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)dyn_smem<MT>());
  });
}

template <int MT>
void allow_smem_dd() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(dd_cg_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem<MT>());
  });
}

template <int MT>
int max_blocks_dd() {
  allow_smem_dd<MT>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dd_cg_kernel<MT>, threads_for<MT>(), dyn_smem<MT>());
  return nb;
}

template <int MT>
cudaError_t launch_dd(const SolverArgs& a, int grid, cudaStream_t st) {
  allow_smem_dd<MT>();
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)dd_cg_kernel<MT>, dim3(grid), dim3(threads_for<MT>()), args,
                                     dyn_smem<MT>(), st);
}

template <int MT, typename T, int VC>
int max_blocks_for() {
  allow_smem<MT, T, VC>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<MT, T, VC>, threads_for<MT>(), dyn_smem<MT>());
  return nb;
}

template <int MT, typename T, int VC>
cudaError_t launch_tpl(const SolverArgs& a, int grid, cudaStream_t st) {
  allow_smem<MT, T, VC>();
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)solve_kernel<MT, T, VC>, dim3(grid), dim3(threads_for<MT>()),
                                     args, dyn_smem<MT>(), st);
}

}  // namespace

int solver_threads(int mt) { return mt == 1 ? threads_for<1>() : threads_for<4>(); }

// One block per SM (the reductions read one partial per block, <= 1024).
int solver_max_grid(int mt, int num_sms) {
  const int nb = (mt == 1) ? std::min(std::min(std::min(max_blocks_for<1, double, 0>(), max_blocks_for<1, float, 0>()),
                                              max_blocks_for<1, double, 1>()),
                                     max_blocks_dd<1>())
                           : std::min(std::min(std::min(max_blocks_for<4, double, 0>(), max_blocks_for<4, float, 0>()),
                                               max_blocks_for<4, double, 1>()),
                                      max_blocks_dd<4>());
  const int g = (nb >= 1) ? num_sms : 0;
  return g > kMaxThreads ? kMaxThreads : g;
}

cudaError_t launch_solver(const SolverArgs& a, int mt, int grid, cudaStream_t st) {
  if (a.df) {  // double-float CG on A (mode 0)
    if (a.mode != 0 || a.fp32 || !a.A.val2 || !a.b || !a.x) return cudaErrorInvalidValue;
    if (mt == 1) return launch_dd<1>(a, grid, st);
    if (mt == 4) return launch_dd<4>(a, grid, st);
    return cudaErrorInvalidValue;
  }
  if (a.mode == 3 || a.mode == 4) {  // V-cycle or polynomial: FP64 outer iteration only
    if (a.fp32) return cudaErrorInvalidValue;
    if (a.mode == 3 && (!a.mg || a.mg_K < 1)) return cudaErrorInvalidValue;
    if (a.mode == 4 && (a.poly.deg < 1 || a.poly.deg > 32 || !a.poly.dinv)) return cudaErrorInvalidValue;
    if (mt == 1) return launch_tpl<1, double, 1>(a, grid, st);
    if (mt == 4) return launch_tpl<4, double, 1>(a, grid, st);
  } else if (a.fp32) {
    if (mt == 1) return launch_tpl<1, float, 0>(a, grid, st);
    if (mt == 4) return launch_tpl<4, float, 0>(a, grid, st);
  } else {
    if (mt == 1) return launch_tpl<1, double, 0>(a, grid, st);
    if (mt == 4) return launch_tpl<4, double, 0>(a, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mmd
