// Vector, sparse and tall-skinny dense kernels (FP64) used around the
// persistent solver: Lanczos re-orthogonalisation (h = V^T M w, f -= V h),
// restart and Ritz recombinations (V Q, V P), the M-QR Gram matrices and the
// Rayleigh quotient S = W^T F of the refinement, level transfers Psi V and
// residual checks.  Every reduction is two-stage with a fixed order so that
// results do not depend on scheduling.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "kernels.h"

namespace mmd {
namespace {

inline int nblk(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  if (b > 65535LL * 16) b = 65535LL * 16;
  return (int)(b < 1 ? 1 : b);
}

__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = v;
}
__global__ void copy_kernel(double* y, const double* x, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = x[i];
}
__global__ void scal_kernel(double* x, int64_t n, double a) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= a;
}
__global__ void axpy_kernel(double* y, const double* x, int64_t n, double a) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// y = A x, SELL-32: one warp per slice of 32 rows, one row per lane, one FMA
// per stored entry (FP64 instructions are scarce on GB300); up to 4 columns
// per pass so a matrix entry is loaded once for 4 right-hand sides.
__global__ void spmv_kernel(Sell A, const double* __restrict__ x, int64_t ldx, double* __restrict__ y,
                            int64_t ldy, int m) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int c0 = 0; c0 < m; c0 += 4) {
    const int mc = (m - c0) < 4 ? (m - c0) : 4;
    for (int64_t sl = gw; sl < A.nslices; sl += nw) {
      const int32_t base = A.ptr[sl], len = A.len[sl];
      const int32_t row = A.row[sl * 32 + lane];
      double acc[4] = {0, 0, 0, 0};
      // chunks of 8 entries: the loads of a chunk, then its gathers, are in
      // flight together; the last chunk is cut by a warp-uniform predicate
      // (len is the slice's), so there is no serial tail.  FMA order per row:
      // CSR order.
      for (int32_t k = 0; k < len; k += 8) {
        double a[8];
        int64_t j[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t o = base + (k + u) * 32 + lane;
          if (k + u < len) {
            a[u] = A.val[o];
            j[u] = A.col[o];
          } else {
            a[u] = 0.0;
            j[u] = 0;
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < mc) {
            double xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xv[u] = (k + u < len) ? x[j[u] + (c0 + c) * ldx] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (k + u < len) acc[c] = fma(a[u], xv[u], acc[c]);
          }
      }
      if (row >= 0)
        for (int c = 0; c < mc; ++c) y[row + (c0 + c) * ldy] = acc[c];
    }
  }
}

// y = A x for one column, SELL-32, one row per lane: chunks of U entries
// whose value and column loads, then gathers, are in flight together (the
// last chunk cut by a warp-uniform predicate, len being the slice's); the
// matrix is streamed once (evict-first loads), x is gathered through the
// cache.  BS threads per block, at least MINB blocks per SM (bounds the
// registers so that enough warps are resident to cover the memory latency).
template <int U, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB)
    spmv1_kernel(Sell A, const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t(blockIdx.x) * BS + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * BS) >> 5;
  for (int64_t sl = gw; sl < A.nslices; sl += nw) {
    const int32_t base = A.ptr[sl] + lane, len = A.len[sl];
    const int32_t row = A.row[sl * 32 + lane];
    double acc = 0.0;
    for (int32_t k = 0; k < len; k += U) {
      double a[U];
      int32_t j[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k + u < len) {
          a[u] = __ldcs(A.val + base + (k + u) * 32);
          j[u] = __ldcs(A.col + base + (k + u) * 32);
        } else {
          a[u] = 0.0;
          j[u] = 0;
        }
      }
      double xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = (k + u < len) ? __ldg(x + j[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k + u < len) acc = fma(a[u], xv[u], acc);
    }
    if (row >= 0) y[row] = acc;
  }
}

struct Spmv1Variant {
  void (*fn)(Sell, const double*, double*);
  int bs, minb;
};
const Spmv1Variant kSpmv1[] = {
    {spmv1_kernel<4, 128, 10>, 128, 10}, {spmv1_kernel<4, 256, 5>, 256, 5},  {spmv1_kernel<8, 128, 8>, 128, 8},
    {spmv1_kernel<8, 256, 4>, 256, 4},   {spmv1_kernel<8, 512, 2>, 512, 2},  {spmv1_kernel<16, 128, 4>, 128, 4},
};
constexpr int kNumSpmv1 = int(sizeof(kSpmv1) / sizeof(kSpmv1[0]));

void launch_spmv1(int v, const Sell& A, const double* x, double* y, cudaStream_t st) {
  const Spmv1Variant& K = kSpmv1[v];
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (A.nslices * 32 + K.bs - 1) / K.bs;
  const int64_t cap = int64_t(nsm) * K.minb * 4;  // a few waves of resident blocks, then a slice-stride loop
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  K.fn<<<(int)blocks, K.bs, 0, st>>>(A, x, y);
}

constexpr int kDotBlocks = 512;

__global__ void dots_stage1(const double* x, const double* y, int64_t n, int64_t ld, int m, double* part) {
  __shared__ double red[32];
  for (int c = 0; c < m; ++c) {
    double s = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
      s = fma(x[i + c * ld], y[i + c * ld], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[size_t(c) * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void dots_stage2(const double* part, int nb, int m, double* out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[size_t(c) * nb + i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[c] = s;
}

// h = B^T u, stage 1: block (row chunk, 32-column group)
constexpr int kGvChunk = 2048;
__global__ void gemv_t_stage1(const double* __restrict__ B, int64_t ldb, int64_t n, int j,
                              const double* __restrict__ u, double* part) {
  __shared__ double us[kGvChunk];
  const int64_t r0 = int64_t(blockIdx.x) * kGvChunk;
  const int rows = (int)((n - r0) < kGvChunk ? (n - r0) : kGvChunk);
  for (int t = threadIdx.x; t < rows; t += blockDim.x) us[t] = u[r0 + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int cc = wid; cc < 32; cc += nw) {
    const int c = blockIdx.y * 32 + cc;
    if (c >= j) break;
    const double* col = B + r0 + c * ldb;
    double s = 0;
    for (int t = lane; t < rows; t += 32) s = fma(col[t], us[t], s);
    s = warp_sum(s);
    if (lane == 0) part[size_t(c) * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void gemv_t_stage2(const double* part, int nchunk, int j, double* h) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= j) return;
  double s = 0;
  for (int i = 0; i < nchunk; ++i) s += part[size_t(c) * nchunk + i];
  h[c] = s;
}

__global__ void gemv_n_kernel(const double* __restrict__ B, int64_t ldb, int64_t n, int j,
                              const double* __restrict__ h, double alpha, double* __restrict__ y) {
  __shared__ double hs[1024];
  for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x; i0 < n; i0 += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    double s = 0;
    for (int c0 = 0; c0 < j; c0 += 1024) {
      const int cn = (j - c0) < 1024 ? (j - c0) : 1024;
      __syncthreads();
      for (int t = threadIdx.x; t < cn; t += blockDim.x) hs[t] = h[c0 + t];
      __syncthreads();
      if (i < n)
        for (int c = 0; c < cn; ++c) s = fma(B[i + (c0 + c) * ldb], hs[c], s);
    }
    if (i < n) y[i] = fma(alpha, s, y[i]);
  }
}

// ---- C = alpha A^T B + beta C (split-K), 64 x 64 tiles, 256 threads (4x4 each)
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void gemm_tn_stage1(int m, int n, int64_t K, int64_t kchunk, const double* __restrict__ A, int64_t lda,
                               const double* __restrict__ B, int64_t ldb, double* part) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int64_t k0 = int64_t(blockIdx.z) * kchunk;
  const int64_t k1 = (k0 + kchunk) < K ? (k0 + kchunk) : K;
  double acc[4][4] = {};
  for (int64_t kk = k0; kk < k1; kk += TK) {
    for (int t = threadIdx.x; t < TK * TM; t += blockDim.x) {
      const int kr = t % TK, ci = t / TK;
      const int64_t k = kk + kr;
      As[kr][ci] = (k < k1 && i0 + ci < m) ? A[k + int64_t(i0 + ci) * lda] : 0.0;
      Bs[kr][ci] = (k < k1 && j0 + ci < n) ? B[k + int64_t(j0 + ci) * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kr = 0; kr < TK; ++kr) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kr][ty + 16 * u];
        b[u] = Bs[kr][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* P = part + size_t(blockIdx.z) * m * n;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, jj = j0 + tx + 16 * v;
      if (i < m && jj < n) P[i + size_t(jj) * m] = acc[u][v];
    }
}
__global__ void gemm_tn_stage2(int m, int n, int nsplit, const double* part, double alpha, double beta, double* C,
                               int64_t ldc) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(m) * n) return;
  const int i = (int)(t % m), jj = (int)(t / m);
  double s = 0;
  for (int z = 0; z < nsplit; ++z) s += part[size_t(z) * m * n + t];
  double* c = C + i + jj * ldc;
  *c = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *c);
}

// ---- C = alpha A B + beta C; A: M x k, B: k x n
__global__ void gemm_nn_kernel(int64_t M, int n, int k, double alpha, const double* __restrict__ A, int64_t lda,
                               const double* __restrict__ B, int64_t ldb, double beta, double* C, int64_t ldc) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t i0 = int64_t(blockIdx.x) * TM;
  const int j0 = blockIdx.y * TN;
  double acc[4][4] = {};
  for (int kk = 0; kk < k; kk += TK) {
    for (int t = threadIdx.x; t < TK * TM; t += blockDim.x) {
      const int ri = t % TM, kr = t / TM;
      As[kr][ri] = (kk + kr < k && i0 + ri < M) ? A[i0 + ri + int64_t(kk + kr) * lda] : 0.0;
      const int kr2 = t % TK, cj = t / TK;
      Bs[kr2][cj] = (kk + kr2 < k && j0 + cj < n) ? B[kk + kr2 + int64_t(j0 + cj) * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kr = 0; kr < TK; ++kr) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kr][ty + 16 * u];
        b[u] = Bs[kr][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t i = i0 + ty + 16 * u;
      const int jj = j0 + tx + 16 * v;
      if (i < M && jj < n) {
        double* c = C + i + int64_t(jj) * ldc;
        *c = (beta == 0.0) ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *c);
      }
    }
}

__global__ void gather_kernel(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y,
                              int64_t ldy) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n * m; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    y[i + c * ldy] = x[perm[i] + c * ldx];
  }
}
__global__ void scatter_kernel(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y,
                               int64_t ldy) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n * m; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    y[perm[i] + c * ldy] = x[i + c * ldx];
  }
}
__global__ void project_kernel(double* x, int64_t ld, int m, const int32_t* seg, const double* phi, int64_t nseg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < nseg * m;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t s = t % nseg, c = t / nseg;
    double* xc = x + c * ld;
    double d = 0;
    for (int32_t i = seg[s]; i < seg[s + 1]; ++i) d = fma(phi[i], xc[i], d);
    for (int32_t i = seg[s]; i < seg[s + 1]; ++i) xc[i] = fma(-phi[i], d, xc[i]);
  }
}
__global__ void scale_cols_kernel(double* x, int64_t ld, int64_t n, int m, const double* s) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n * m; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    x[i + c * ld] *= s[c];
  }
}

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void random_kernel(double* x, int64_t n, uint64_t seed, uint64_t stream, const int32_t* perm) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const uint64_t key = splitmix_mix(seed + (stream + 1) * G);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t idx = perm ? (uint64_t)perm[i] : (uint64_t)i;
    const uint64_t bits = splitmix_mix(key + (idx + 1) * G);
    x[i] = 2.0 * (double)(bits >> 11) * 0x1.0p-53 - 1.0;
  }
}

// one block per column: normalise to unit 2-norm, largest-|.| entry positive (lowest index on ties)
__global__ void normalise_sign_kernel(double* V, int64_t ld, int64_t n) {
  __shared__ double red[32];
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  double* v = V + int64_t(blockIdx.x) * ld;
  double s = 0, best = -1;
  int64_t besti = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = v[i];
    s = fma(a, a, s);
    if (fabs(a) > best) {
      best = fabs(a);
      besti = i;
    }
  }
  s = block_sum(s, red);
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = bv[threadIdx.x + o];
      const int64_t i2 = bi[threadIdx.x + o];
      if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = b2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const double sc = (v[bi[0]] < 0 ? -1.0 : 1.0) / sqrt(s);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] *= sc;
}

__global__ void resid_stage1(const double* Y, const double* V, int64_t ld, int64_t n, int m, const double* lam,
                             double* part) {
  // Y has leading dimension n, V has ld
  __shared__ double red[32];
  for (int c = 0; c < m; ++c) {
    double s = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
      const double t = Y[i + c * n] - lam[c] * V[i + c * ld];
      s = fma(t, t, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[size_t(c) * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void sqrt_kernel(double* x, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) x[i] = sqrt(x[i]);
}

}  // namespace

__global__ void sub_kernel(double* r, const double* b, const double* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    r[i] = b[i] - y[i];
}
__global__ void to_f32_kernel(float* f, const double* d, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    f[i] = (float)d[i];
}
__global__ void add_f32_kernel(double* x, const float* f, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] += (double)f[i];
}

void k_sub(double* r, const double* b, const double* y, int64_t n, cudaStream_t st) {
  sub_kernel<<<nblk(n, 256), 256, 0, st>>>(r, b, y, n);
}
void k_to_f32(float* f, const double* d, int64_t n, cudaStream_t st) {
  to_f32_kernel<<<nblk(n, 256), 256, 0, st>>>(f, d, n);
}
void k_add_f32(double* x, const float* f, int64_t n, cudaStream_t st) {
  add_f32_kernel<<<nblk(n, 256), 256, 0, st>>>(x, f, n);
}

void k_fill(double* x, int64_t n, double v, cudaStream_t st) { fill_kernel<<<nblk(n, 256), 256, 0, st>>>(x, n, v); }
void k_copy(double* y, const double* x, int64_t n, cudaStream_t st) {
  copy_kernel<<<nblk(n, 256), 256, 0, st>>>(y, x, n);
}
void k_scal(double* x, int64_t n, double a, cudaStream_t st) { scal_kernel<<<nblk(n, 256), 256, 0, st>>>(x, n, a); }
void k_axpy(double* y, const double* x, int64_t n, double a, cudaStream_t st) {
  axpy_kernel<<<nblk(n, 256), 256, 0, st>>>(y, x, n, a);
}

void k_spmv(const Sell& A, const double* x, int64_t ldx, double* y, int64_t ldy, int m, cudaStream_t st) {
  if (m == 1 && A.variant >= 0 && A.variant < kNumSpmv1) {
    launch_spmv1(A.variant, A, x, y, st);
    return;
  }
  const int threads = 256;
  int64_t blocks = (A.nslices * 32 + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  spmv_kernel<<<(int)blocks, threads, 0, st>>>(A, x, ldx, y, ldy, m);
}

int k_spmv_variants() { return kNumSpmv1; }

int k_spmv_autotune(const Sell& A, const double* x, double* y, cudaStream_t st, float* ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1;
  }
  int best = -1;
  float best_ms = 0.f;
  for (int v = 0; v < kNumSpmv1; ++v) {
    launch_spmv1(v, A, x, y, st);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) launch_spmv1(v, A, x, y, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      best = -1;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 5.f;
    if (ms_out) ms_out[v] = ms;
    if (best < 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void k_dots(const double* x, const double* y, int64_t n, int64_t ld, int m, double* out, double* scratch,
            cudaStream_t st) {
  int nb = (int)((n + 255) / 256);
  if (nb > kDotBlocks) nb = kDotBlocks;
  if (nb < 1) nb = 1;
  dots_stage1<<<nb, 256, 0, st>>>(x, y, n, ld, m, scratch);
  dots_stage2<<<m, 256, 0, st>>>(scratch, nb, m, out);
}

void k_gemv_t(const double* B, int64_t ldb, int64_t n, int j, const double* u, double* h, double* scratch,
              cudaStream_t st) {
  if (j <= 0) return;
  const int nchunk = (int)((n + kGvChunk - 1) / kGvChunk);
  dim3 g(nchunk, (j + 31) / 32);
  gemv_t_stage1<<<g, 256, 0, st>>>(B, ldb, n, j, u, scratch);
  gemv_t_stage2<<<(j + 127) / 128, 128, 0, st>>>(scratch, nchunk, j, h);
}

void k_gemv_n(const double* B, int64_t ldb, int64_t n, int j, const double* h, double alpha, double* y,
              cudaStream_t st) {
  if (j <= 0) return;
  gemv_n_kernel<<<nblk(n, 256), 256, 0, st>>>(B, ldb, n, j, h, alpha, y);
}

void k_gemm_tn(int m, int n, int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, double* scratch, int64_t scratch_len, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  const int tiles = ((m + TM - 1) / TM) * ((n + TN - 1) / TN);
  int64_t nsplit = (4 * 152 + tiles - 1) / tiles;
  const int64_t maxsplit = (K + 255) / 256;
  if (nsplit > maxsplit) nsplit = maxsplit;
  const int64_t cap = scratch_len / (int64_t(m) * n);
  if (cap < 1) return;  // caller guarantees scratch_len >= m * n
  if (nsplit > cap) nsplit = cap;
  if (nsplit < 1) nsplit = 1;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  dim3 g((m + TM - 1) / TM, (n + TN - 1) / TN, (unsigned)nsplit);
  gemm_tn_stage1<<<g, 256, 0, st>>>(m, n, K, kchunk, A, lda, B, ldb, scratch);
  const int64_t tot = int64_t(m) * n;
  gemm_tn_stage2<<<(int)((tot + 255) / 256), 256, 0, st>>>(m, n, (int)nsplit, scratch, alpha, beta, C, ldc);
}

void k_gemm_nn(int64_t M, int n, int k, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, cudaStream_t st) {
  if (M <= 0 || n <= 0) return;
  dim3 g((unsigned)((M + TM - 1) / TM), (n + TN - 1) / TN);
  gemm_nn_kernel<<<g, 256, 0, st>>>(M, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

void k_gather(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y, int64_t ldy,
              cudaStream_t st) {
  gather_kernel<<<nblk(n * m, 256), 256, 0, st>>>(x, ldx, perm, n, m, y, ldy);
}
void k_scatter(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y, int64_t ldy,
               cudaStream_t st) {
  scatter_kernel<<<nblk(n * m, 256), 256, 0, st>>>(x, ldx, perm, n, m, y, ldy);
}
void k_project(double* x, int64_t ld, int m, const int32_t* seg_ptr, const double* phi, int64_t nseg,
               cudaStream_t st) {
  project_kernel<<<nblk(nseg * m, 256), 256, 0, st>>>(x, ld, m, seg_ptr, phi, nseg);
}
void k_scale_cols(double* x, int64_t ld, int64_t n, int m, const double* s, cudaStream_t st) {
  scale_cols_kernel<<<nblk(n * m, 256), 256, 0, st>>>(x, ld, n, m, s);
}
void k_random(double* x, int64_t n, uint64_t seed, uint64_t stream, const int32_t* perm, cudaStream_t st) {
  random_kernel<<<nblk(n, 256), 256, 0, st>>>(x, n, seed, stream, perm);
}
void k_normalise_sign(double* V, int64_t ld, int64_t n, int m, double* scratch, cudaStream_t st) {
  (void)scratch;
  if (m > 0) normalise_sign_kernel<<<m, 1024, 0, st>>>(V, ld, n);
}
void k_residuals(const Sell& A, int64_t n, const double* V, int64_t ld, int m, const double* lam, double* out,
                 double* scratch, cudaStream_t st) {
  // scratch: n*m (A V) + 512*m partials
  double* Y = scratch;
  double* part = scratch + n * m;
  k_spmv(A, V, ld, Y, n, m, st);
  int nb = (int)((n + 255) / 256);
  if (nb > kDotBlocks) nb = kDotBlocks;
  resid_stage1<<<nb, 256, 0, st>>>(Y, V, ld, n, m, lam, part);
  dots_stage2<<<m, 256, 0, st>>>(part, nb, m, out);
  sqrt_kernel<<<(m + 127) / 128, 128, 0, st>>>(out, m);
}

}  // namespace mmd

namespace mmd {
namespace {
// G[e] = sum_i U(r_e, i) V(c_e, i) for the stored entries e of a CSR pattern
// (sampled dense-dense product); one warp per row, one lane per entry.
__global__ void sddmm_kernel(const int32_t* rp, const int32_t* ci, int64_t n, const double* U, const double* V,
                             int64_t ld, int N, double* G) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n;
       r += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    for (int32_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
      const int64_t c = ci[e];
      double s = 0.0;
      for (int i = 0; i < N; ++i) s = fma(U[r + i * ld], V[c + i * ld], s);
      G[e] = s;
    }
  }
}
}  // namespace

void k_sddmm(const int32_t* rp, const int32_t* ci, int64_t n, const double* U, const double* V, int64_t ld, int N,
             double* G, cudaStream_t st) {
  int64_t b = (n * 32 + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  sddmm_kernel<<<(int)b, 256, 0, st>>>(rp, ci, n, U, V, ld, N, G);
}
}  // namespace mmd
