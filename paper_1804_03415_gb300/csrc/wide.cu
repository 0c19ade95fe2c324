// Many right-hand sides of one level-0 solve in one persistent launch: the
// block of warm-started solves A F = W of the refinement (Algorithm 5, every
// column its own CG recurrence, M^(0) = I), m columns at once.
//
// Layout: the solver's vectors are row-major n x m (element (i, c) at
// i m + c), so the gather of one matrix entry's row X(j, :) is one contiguous
// run of m values; a warp takes one row of A at a time, its lanes two columns
// each (64 per pass), the row's entries read eight at a time by eight lanes
// and broadcast by shuffles.  Arithmetic is double-float (pairs of FP32
// numbers, about 48 bits; Dekker 1971, Knuth's two-sum and the FMA
// two-product), FP32 issue being about seventy times the FP64 rate on this
// GPU; the scalars alpha, beta stay FP64 and a column is accepted only when
// its FP64 residual b - A x meets the tolerance (at most three restarts from
// x with that residual while it falls; a column that stalls is reported
// unconverged and finished by the caller in FP64).  The recurrence is
// Chronopoulos-Gear CG: one reduction round and one plain grid barrier per
// iteration for all columns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kernels.h"

namespace mmd {

namespace {

constexpr int kWT = 768;        // threads per block, one block per SM
constexpr int kWW = kWT / 32;   // warps per block
constexpr int kU = 8;           // entries of a row read per chunk

struct pd {
  float hi, lo;
};
__device__ __forceinline__ pd pd_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double pd_val(pd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ pd pd_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ pd pd_add(pd a, pd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return pd_renorm(s, e);
}
__device__ __forceinline__ pd pd_fma(pd a, pd b, pd c) {  // a b + c
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  return pd_renorm(s, e);
}

__device__ __forceinline__ int64_t wlo(int64_t n) { return n * blockIdx.x / gridDim.x; }
__device__ __forceinline__ int64_t whi(int64_t n) { return n * (blockIdx.x + 1) / gridDim.x; }

struct WideSh {
  double rz[kWideMaxCols], alpha[kWideMaxCols], bn[kWideMaxCols], tr[kWideMaxCols], last[kWideMaxCols];
  int act[kWideMaxCols], ok[kWideMaxCols], msk[kWideMaxCols];
  long long it[kWideMaxCols], base[kWideMaxCols];
  float2 al[kWideMaxCols], be[kWideMaxCols];
  union {
    struct {
      float2 pa[kWW][64], pb[kWW][64];
    } f;
    double qa[kWW][64];
  } u;
};

// Per-column sums of one 64-column chunk, held per lane (columns cb + lane and
// cb + 32 + lane) by every warp: block sums into red[slot][c][block].
__device__ __forceinline__ void chunk_partials_pd(WideSh& s, float2* red, int slot, int m, int cb, pd a0, pd a1,
                                                  int slot2, pd b0, pd b1) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  s.u.f.pa[w][lane] = make_float2(a0.hi, a0.lo);
  s.u.f.pa[w][32 + lane] = make_float2(a1.hi, a1.lo);
  s.u.f.pb[w][lane] = make_float2(b0.hi, b0.lo);
  s.u.f.pb[w][32 + lane] = make_float2(b1.hi, b1.lo);
  __syncthreads();
  if (threadIdx.x < 64) {
    const int c = cb + threadIdx.x;
    if (c < m) {
      pd ta = {0.f, 0.f}, tb = {0.f, 0.f};
      for (int q = 0; q < kWW; ++q) {
        ta = pd_add(ta, {s.u.f.pa[q][threadIdx.x].x, s.u.f.pa[q][threadIdx.x].y});
        tb = pd_add(tb, {s.u.f.pb[q][threadIdx.x].x, s.u.f.pb[q][threadIdx.x].y});
      }
      red[(size_t(slot) * m + c) * gridDim.x + blockIdx.x] = make_float2(ta.hi, ta.lo);
      red[(size_t(slot2) * m + c) * gridDim.x + blockIdx.x] = make_float2(tb.hi, tb.lo);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void chunk_partials_f64(WideSh& s, double* red, int m, int cb, double a0, double a1) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  s.u.qa[w][lane] = a0;
  s.u.qa[w][32 + lane] = a1;
  __syncthreads();
  if (threadIdx.x < 64) {
    const int c = cb + threadIdx.x;
    if (c < m) {
      double t = 0.0;
      for (int q = 0; q < kWW; ++q) t += s.u.qa[q][threadIdx.x];
      red[size_t(c) * gridDim.x + blockIdx.x] = t;
    }
  }
  __syncthreads();
}

// r = b - A x in FP64 for the columns with mask[c] (x from the pairs xd, or 0
// with first), stored as pairs; dst[c] = ||r_c||^2; also ||b_c||^2 into
// bnorm when it is not NULL.  x64 (row-major FP64 scratch) receives x.
__device__ bool wide_true_residual(const WideArgs& a, WideSh& s, const int* mask, bool first, double* dst,
                                   double* bnorm) {
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  const pd* xd = (const pd*)a.xd;
  pd* r = (pd*)a.r;
  double* x64 = a.q64;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!first) {
    for (int64_t i = wlo(n) + w; i < whi(n); i += kWW)
      for (int c = lane; c < m; c += 32) {
        const double v = pd_val(xd[i * m + c]);
        x64[i * m + c] = v;
        a.x[i + c * ld] = v;
      }
    if (!grid_sync(a.bar)) return false;
  }
  for (int cb = 0; cb < m; cb += 64) {
    const int c0 = cb + lane, c1 = cb + 32 + lane;
    const bool on0 = c0 < m && mask[c0], on1 = c1 < m && mask[c1];
    double q0 = 0.0, q1 = 0.0, b0 = 0.0, b1 = 0.0;
    for (int64_t i = wlo(n) + w; i < whi(n); i += kWW) {
      double s0 = 0.0, s1 = 0.0;
      if (!first) {
        const int32_t e0 = a.rowptr[i], e1 = a.rowptr[i + 1];
        for (int32_t kb = e0; kb < e1; kb += 32) {
          const int cnt = min(32, e1 - kb);
          double av = 0.0;
          int jj = 0;
          if (lane < cnt) {
            av = a.val[kb + lane];
            jj = a.col[kb + lane];
          }
          for (int u = 0; u < cnt; ++u) {
            const double au = __shfl_sync(0xffffffffu, av, u);
            const int j = __shfl_sync(0xffffffffu, jj, u);
            if (on0) s0 = fma(au, x64[size_t(j) * m + c0], s0);
            if (on1) s1 = fma(au, x64[size_t(j) * m + c1], s1);
          }
        }
      }
      if (on0) {
        const double bv = a.b[i + c0 * ld], rv = bv - s0;
        r[i * m + c0] = pd_of(rv);
        q0 = fma(rv, rv, q0);
        b0 = fma(bv, bv, b0);
      }
      if (on1) {
        const double bv = a.b[i + c1 * ld], rv = bv - s1;
        r[i * m + c1] = pd_of(rv);
        q1 = fma(rv, rv, q1);
        b1 = fma(bv, bv, b1);
      }
    }
    chunk_partials_f64(s, a.red64, m, cb, q0, q1);
    if (bnorm) chunk_partials_f64(s, a.red64 + size_t(m) * gridDim.x, m, cb, b0, b1);
  }
  if (!grid_sync(a.bar)) return false;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double t = 0.0, tb = 0.0;
    for (int g = 0; g < (int)gridDim.x; ++g) {
      t += a.red64[size_t(c) * gridDim.x + g];
      if (bnorm) tb += a.red64[(size_t(m) + c) * gridDim.x + g];
    }
    if (mask[c]) dst[c] = t;
    if (bnorm) bnorm[c] = tb;
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kWT, 1) wide_cg_kernel(WideArgs a) {
  __shared__ WideSh s;
  grid_sync_init();
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  pd* const r = (pd*)a.r;
  pd* const p = (pd*)a.p;
  pd* const sv = (pd*)a.s;
  pd* const w = (pd*)a.w;
  pd* const xd = (pd*)a.xd;
  float2* const red2 = (float2*)a.red;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the iterate as pairs (x0 or 0)
  for (int64_t i = wlo(n) + warp; i < whi(n); i += kWW)
    for (int c = lane; c < m; c += 32) {
      if (a.x0) {
        xd[i * m + c] = pd_of(a.x[i + c * ld]);
      } else {
        xd[i * m + c] = {0.f, 0.f};
        a.x[i + c * ld] = 0.0;
      }
    }
  for (int c = threadIdx.x; c < m; c += blockDim.x) s.act[c] = 1;
  __syncthreads();
  if (!grid_sync(a.bar)) return;
  if (!wide_true_residual(a, s, s.act, !a.x0, s.tr, s.bn)) return;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    s.bn[c] = sqrt(s.bn[c]);
    s.rz[c] = s.tr[c];
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.tr[c]) <= a.tol * s.bn[c]);
    s.ok[c] = !s.act[c];
    s.it[c] = 0;
    s.last[c] = sqrt(s.tr[c]);
  }
  __syncthreads();
  for (int pass = 0;; ++pass) {
    for (int c = threadIdx.x; c < m; c += blockDim.x) s.base[c] = s.it[c];
    __syncthreads();
    for (int it = 1;; ++it) {
      int any = 0;
      for (int c = 0; c < m; ++c) any |= (s.act[c] == 1);
      if (!any) break;
      // w = A r, delta = r^T w, gamma = r^T r, for the running columns
      for (int cb = 0; cb < m; cb += 64) {
        const int c0 = cb + lane, c1 = cb + 32 + lane;
        const bool on0 = c0 < m && s.act[c0] == 1, on1 = c1 < m && s.act[c1] == 1;
        pd d0 = {0.f, 0.f}, d1 = {0.f, 0.f}, g0 = {0.f, 0.f}, g1 = {0.f, 0.f};
        if (__any_sync(0xffffffffu, on0 || on1)) {
          for (int64_t i = wlo(n) + warp; i < whi(n); i += kWW) {
            const int32_t e0 = a.rowptr[i], e1 = a.rowptr[i + 1];
            pd acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
            for (int32_t kb = e0; kb < e1; kb += kU) {
              const int cnt = min(kU, e1 - kb);
              float ah = 0.f, alo = 0.f;
              int jj = 0;
              if (lane < cnt) {
                const float2 v = a.val2[kb + lane];
                ah = v.x;
                alo = v.y;
                jj = a.col[kb + lane];
              }
              pd x0v[kU], x1v[kU];
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const int j = __shfl_sync(0xffffffffu, jj, u);
                x0v[u] = {0.f, 0.f};
                x1v[u] = {0.f, 0.f};
                if (u < cnt) {
                  if (on0) x0v[u] = r[size_t(j) * m + c0];
                  if (on1) x1v[u] = r[size_t(j) * m + c1];
                }
              }
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const pd au = {__shfl_sync(0xffffffffu, ah, u), __shfl_sync(0xffffffffu, alo, u)};
                if (u < cnt) {
                  if (on0) acc0 = pd_fma(au, x0v[u], acc0);
                  if (on1) acc1 = pd_fma(au, x1v[u], acc1);
                }
              }
            }
            if (on0) {
              const pd rv = r[i * m + c0];
              w[i * m + c0] = acc0;
              d0 = pd_fma(rv, acc0, d0);
              g0 = pd_fma(rv, rv, g0);
            }
            if (on1) {
              const pd rv = r[i * m + c1];
              w[i * m + c1] = acc1;
              d1 = pd_fma(rv, acc1, d1);
              g1 = pd_fma(rv, rv, g1);
            }
          }
        }
        chunk_partials_pd(s, red2, 0, m, cb, d0, d1, 1, g0, g1);
      }
      if (!grid_sync(a.bar)) return;
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        if (s.act[c] != 1) continue;
        pd td = {0.f, 0.f}, tg = {0.f, 0.f};
        for (int g = 0; g < (int)gridDim.x; ++g) {
          const float2 u = red2[size_t(c) * gridDim.x + g], v = red2[(size_t(m) + c) * gridDim.x + g];
          td = pd_add(td, {u.x, u.y});
          tg = pd_add(tg, {v.x, v.y});
        }
        const double dl = pd_val(td), gm = pd_val(tg);
        if (it > 1 && gm <= a.tol * a.tol * s.bn[c] * s.bn[c]) {
          s.act[c] = 2;  // the recurrence converged after update it - 1: check the true residual
        } else if (s.base[c] + it <= a.maxit) {
          double be = 0.0, den = dl;
          if (it > 1) {
            be = gm / s.rz[c];
            den = dl - be * gm / s.alpha[c];
          }
          if (!(den > 0.0)) {
            s.act[c] = 0;  // not SPD at this precision: finished by the caller in FP64
          } else {
            s.rz[c] = gm;
            s.alpha[c] = gm / den;
            const pd al = pd_of(s.alpha[c]), bt = pd_of(be);
            s.al[c] = make_float2(al.hi, al.lo);
            s.be[c] = make_float2(bt.hi, bt.lo);
            s.it[c] = s.base[c] + it;
          }
        } else {
          s.act[c] = 0;  // iteration cap
        }
      }
      __syncthreads();
      // p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s
      const bool first = (it == 1);
      for (int64_t i = wlo(n) + warp; i < whi(n); i += kWW)
        for (int c = lane; c < m; c += 32) {
        if (s.act[c] != 1) continue;
        const int64_t f = i * m + c;
        const pd al = {s.al[c].x, s.al[c].y}, be = {s.be[c].x, s.be[c].y};
        const pd rv = r[f], wv = w[f];
        const pd pv = first ? rv : pd_fma(be, p[f], rv);
        const pd svv = first ? wv : pd_fma(be, sv[f], wv);
        p[f] = pv;
        sv[f] = svv;
        xd[f] = pd_fma(al, pv, xd[f]);
        r[f] = pd_fma({-al.hi, -al.lo}, svv, rv);
      }
      if (!grid_sync(a.bar)) return;
    }
    // FP64 residual of the columns whose recurrence converged; x written out
    int chk_any = 0;
    for (int c = 0; c < m; ++c) chk_any |= (s.act[c] == 2);
    if (!chk_any) {
      for (int64_t i = wlo(n) + warp; i < whi(n); i += kWW)
        for (int c = lane; c < m; c += 32) a.x[i + c * ld] = pd_val(xd[i * m + c]);
      break;
    }
    for (int c = threadIdx.x; c < m; c += blockDim.x) s.msk[c] = (s.act[c] == 2);
    __syncthreads();
    if (!wide_true_residual(a, s, s.msk, false, s.tr, nullptr)) return;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      if (!s.msk[c]) continue;
      const double tn = sqrt(s.tr[c]);
      if (tn <= a.tol * s.bn[c]) {
        s.act[c] = 0;
        s.ok[c] = 1;
      } else if (pass < 3 && tn < 0.5 * s.last[c]) {
        s.act[c] = 1;
        s.rz[c] = s.tr[c];
        s.last[c] = tn;
      } else {
        s.act[c] = 0;
      }
    }
    __syncthreads();
    int again = 0;
    for (int c = 0; c < m; ++c) again |= (s.act[c] == 1);
    if (!again) break;
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      a.it_out[c] = s.it[c];
      a.conv[c] = s.ok[c];
    }
}

}  // namespace

int wide_max_grid(int num_sms) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wide_cg_kernel, kWT, 0);
  return nb >= 1 ? num_sms : 0;
}

cudaError_t launch_wide_cg(const WideArgs& a, int grid, cudaStream_t st) {
  if (a.m < 1 || a.m > kWideMaxCols || !a.val2 || !a.val || !a.b || !a.x || grid < 1) return cudaErrorInvalidValue;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)wide_cg_kernel, dim3(grid), dim3(kWT), args, 0, st);
}

}  // namespace mmd
