// Persistent CG / flexible-PCG kernel: the inner loop of Operator OP
// (Section 4: y = pcg(A^(k), M^(k) x, M^(k), 0, eps), with M^(k)^{-1} applied
// by an inner CG to 0.1 eps) and of the two solves of the Eigenpair
// Refinement (Algorithm 5: CG on B^(l) = U^T A U and the warm-started PCG).
//
// One cooperative launch runs a whole solve for m <= MT right-hand sides
// (column-major, leading dimension ld).  Every block owns rows in a strided
// pattern; a group of TPR lanes computes one CSR row (vector CSR SpMV) and the
// dot products of the iteration are fused into the SpMV and the vector
// updates.  Scalars never leave the device: each block writes its partial
// sums, a bounded grid barrier follows, and every block then reduces the same
// partials in the same order, so all blocks take identical decisions.
//
// Modes
//   0  CG on A (M = I; the paper's pcg(A, b, -, x0, eps))
//   1  flexible PCG on A with preconditioner M applied by an inner CG;
//      beta = z+^T (r+ - r) / (r^T z)  (Golub and Ye, 1999), computed as
//      -alpha z+^T q / (r^T z) since r+ - r = -alpha q.
//   2  CG on P A P with P = I - Phi Phi^T applied segment by segment.  Since
//      U of Section 2.3 has orthonormal columns and U U^T = P on each patch,
//      this is CG on B = U^T A U in the coordinates U g (same iterates); the
//      solution returned is x = U g.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "kernels.h"

namespace mmd {

namespace {

constexpr int kThreads = 512;

template <int MT>
struct Sh {
  double red[32];
  double bn[MT], rz[MT], rr[MT], alpha[MT], val[MT], val2[MT];
  double irr[MT], irn0[MT], ia[MT];
  int act[MT], iact[MT];
  long long it[MT], iit[MT];
};

// Reduce partial sums red[slot][c][block] -> dst[c] in every block.
template <int MT>
__device__ void reduce_slot(const double* red, int slot, int m, double* dst, double* sred) {
  const int G = gridDim.x;
  for (int c = 0; c < m; ++c) {
    double v = (threadIdx.x < G) ? red[(size_t(slot) * MT + c) * G + threadIdx.x] : 0.0;
    v = block_sum(v, sred);
    if (threadIdx.x == 0) dst[c] = v;
  }
  __syncthreads();
}

template <int MT>
__device__ void write_partials(double* red, int slot, int m, const double* acc, double* sred) {
  for (int c = 0; c < m; ++c) {
    double v = block_sum(acc[c], sred);
    if (threadIdx.x == 0) red[(size_t(slot) * MT + c) * gridDim.x + blockIdx.x] = v;
  }
}

// y(:,c) = A x(:,c) for columns with mask[c]; optionally dacc[c] += w(:,c)^T y(:,c).
template <int TPR, int MT>
__device__ void spmv_cols(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ va, int64_t n, const double* __restrict__ X,
                          double* __restrict__ Y, int64_t ld, int m, const int* mask,
                          const double* __restrict__ W, double* dacc) {
  const int lane = threadIdx.x % TPR;
  const int64_t g = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / TPR;
  const int64_t Gs = (int64_t(gridDim.x) * blockDim.x) / TPR;
  for (int64_t base = 0;; base += Gs) {
    const int64_t i = g + base;
    if (!__any_sync(0xffffffffu, i < n)) break;
    double acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    if (i < n) {
      const int32_t k0 = rp[i], k1 = rp[i + 1];
      for (int32_t k = k0 + lane; k < k1; k += TPR) {
        const double a = va[k];
        const int64_t j = ci[k];
#pragma unroll
        for (int c = 0; c < MT; ++c)
          if (c < m && mask[c]) acc[c] = fma(a, X[j + c * ld], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = group_sum<TPR>(acc[c]);
    if (i < n && lane == 0) {
#pragma unroll
      for (int c = 0; c < MT; ++c)
        if (c < m && mask[c]) {
          Y[i + c * ld] = acc[c];
          if (W) dacc[c] = fma(W[i + c * ld], acc[c], dacc[c]);
        }
    }
  }
}

template <int TPR, int MT>
__device__ bool inner_cg(const SolverArgs& a, Sh<MT>& s, int64_t tid, int64_t nthr) {
  // z = M^{-1} r for active columns, CG to relative residual itol (zero start).
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  double acc[MT];
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
        const double rv = a.r[i + c * ld];
        a.z[i + c * ld] = 0.0;
        a.ir[i + c * ld] = rv;
        a.ip[i + c * ld] = rv;
      }
  if (!grid_sync(a.bar)) return false;
  for (int j = 1; j <= a.imaxit; ++j) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.iact[c];
    if (!any) break;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    spmv_cols<TPR, MT>(a.mrp, a.mcol, a.mval, n, a.ip, a.iq, ld, m, s.iact, a.ip, acc);
    write_partials<MT>(a.red, 2, m, acc, s.red);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 2, m, s.val, s.red);
    if (threadIdx.x < m) s.ia[threadIdx.x] = s.iact[threadIdx.x] ? s.irr[threadIdx.x] / s.val[threadIdx.x] : 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.iact[c]) {
          const int64_t o = i + c * ld;
          a.z[o] = fma(s.ia[c], a.ip[o], a.z[o]);
          const double rv = fma(-s.ia[c], a.iq[o], a.ir[o]);
          a.ir[o] = rv;
          acc[c] = fma(rv, rv, acc[c]);
        }
    write_partials<MT>(a.red, 3, m, acc, s.red);
    if (!grid_sync(a.bar)) return false;
    reduce_slot<MT>(a.red, 3, m, s.val, s.red);
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
          a.ip[o] = fma(s.ia[c], a.ip[o], a.ir[o]);
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

template <int TPR, int MT>
__global__ void __launch_bounds__(kThreads) solve_kernel(SolverArgs a) {
  __shared__ Sh<MT> s;
  const int m = a.m;
  const int64_t n = a.n, ld = a.ld;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  double acc[MT], acc2[MT];
  int all1[MT];
#pragma unroll
  for (int c = 0; c < MT; ++c) all1[c] = 1;
  // ---- set-up: r = b - A x0 (or b), norms
  if (a.x0) spmv_cols<TPR, MT>(a.arp, a.acol, a.aval, n, a.x, a.q, ld, m, all1, nullptr, nullptr);
#pragma unroll
  for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = 0.0;
  if (a.x0 && !grid_sync(a.bar)) return;  // q complete is only needed locally, but keep phases aligned
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c) {
      const int64_t o = i + c * ld;
      const double bv = a.b[o];
      double rv = bv;
      if (a.x0) rv -= a.q[o];
      else a.x[o] = 0.0;
      a.r[o] = rv;
      acc[c] = fma(bv, bv, acc[c]);
      acc2[c] = fma(rv, rv, acc2[c]);
    }
  write_partials<MT>(a.red, 0, m, acc, s.red);
  write_partials<MT>(a.red, 1, m, acc2, s.red);
  if (!grid_sync(a.bar)) return;
  reduce_slot<MT>(a.red, 0, m, s.bn, s.red);
  reduce_slot<MT>(a.red, 1, m, s.rr, s.red);
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    s.bn[c] = sqrt(s.bn[c]);
    s.act[c] = (s.bn[c] > 0.0) && !(sqrt(s.rr[c]) <= a.tol * s.bn[c]);
    s.it[c] = 0;
  }
  __syncthreads();
  for (int64_t i = tid; i < n; i += nthr)  // zero right-hand sides give x = 0
    for (int c = 0; c < m; ++c)
      if (s.bn[c] == 0.0) a.x[i + c * ld] = 0.0;
  double* zv = a.r;
  if (a.mode == 1) {
    if (!inner_cg<TPR, MT>(a, s, tid, nthr)) return;
    zv = a.z;
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    for (int64_t i = tid; i < n; i += nthr)
      for (int c = 0; c < m; ++c)
        if (s.act[c]) acc[c] = fma(a.r[i + c * ld], a.z[i + c * ld], acc[c]);
    write_partials<MT>(a.red, 0, m, acc, s.red);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 0, m, s.rz, s.red);
  } else {
    if (threadIdx.x < m) s.rz[threadIdx.x] = s.rr[threadIdx.x];
    __syncthreads();
  }
  for (int64_t i = tid; i < n; i += nthr)
    for (int c = 0; c < m; ++c)
      if (s.act[c]) a.p[i + c * ld] = zv[i + c * ld];
  if (!grid_sync(a.bar)) return;

  for (int it = 1; it <= a.maxit; ++it) {
    int any = 0;
    for (int c = 0; c < m; ++c) any |= s.act[c];
    if (!any) break;
    // q = A p, p^T q
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    spmv_cols<TPR, MT>(a.arp, a.acol, a.aval, n, a.p, a.q, ld, m, s.act, a.p, acc);
    write_partials<MT>(a.red, 0, m, acc, s.red);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 0, m, s.val, s.red);
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
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    if (a.mode == 2) {
      for (int64_t sg = tid; sg < a.nseg; sg += nthr) {
        const int32_t s0 = a.seg_ptr[sg], s1 = a.seg_ptr[sg + 1];
        for (int c = 0; c < m; ++c) {
          if (!s.act[c]) continue;
          double t = 0.0;
          for (int32_t i = s0; i < s1; ++i) t = fma(a.phi[i], a.q[i + c * ld], t);
          for (int32_t i = s0; i < s1; ++i) {
            const int64_t o = i + c * ld;
            const double qv = fma(-a.phi[i], t, a.q[o]);
            a.x[o] = fma(s.alpha[c], a.p[o], a.x[o]);
            const double rv = fma(-s.alpha[c], qv, a.r[o]);
            a.r[o] = rv;
            acc[c] = fma(rv, rv, acc[c]);
          }
        }
      }
    } else {
      for (int64_t i = tid; i < n; i += nthr)
        for (int c = 0; c < m; ++c)
          if (s.act[c]) {
            const int64_t o = i + c * ld;
            a.x[o] = fma(s.alpha[c], a.p[o], a.x[o]);
            const double rv = fma(-s.alpha[c], a.q[o], a.r[o]);
            a.r[o] = rv;
            acc[c] = fma(rv, rv, acc[c]);
          }
    }
    write_partials<MT>(a.red, 1, m, acc, s.red);
    if (!grid_sync(a.bar)) return;
    reduce_slot<MT>(a.red, 1, m, s.val2, s.red);
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
      if (!inner_cg<TPR, MT>(a, s, tid, nthr)) return;
#pragma unroll
      for (int c = 0; c < MT; ++c) acc[c] = acc2[c] = 0.0;
      for (int64_t i = tid; i < n; i += nthr)
        for (int c = 0; c < m; ++c)
          if (s.act[c]) {
            const int64_t o = i + c * ld;
            acc[c] = fma(a.r[o], a.z[o], acc[c]);
            acc2[c] = fma(a.z[o], a.q[o], acc2[c]);
          }
      write_partials<MT>(a.red, 0, m, acc, s.red);
      write_partials<MT>(a.red, 1, m, acc2, s.red);
      if (!grid_sync(a.bar)) return;
      reduce_slot<MT>(a.red, 0, m, s.val, s.red);
      reduce_slot<MT>(a.red, 1, m, s.val2, s.red);
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
          a.p[o] = fma(s.alpha[c], a.p[o], zv[o]);
        }
    if (!grid_sync(a.bar)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x < m) {
    const int c = threadIdx.x;
    a.it_out[c] = s.it[c];
    a.conv[c] = s.act[c] ? 0 : 1;
  }
}

template <int TPR, int MT>
int max_blocks_for() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<TPR, MT>, kThreads, 0);
  return nb;
}

template <int TPR, int MT>
cudaError_t launch_tpl(const SolverArgs& a, int grid, cudaStream_t st) {
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)solve_kernel<TPR, MT>, dim3(grid), dim3(kThreads), args, 0, st);
}

}  // namespace

int solver_threads() { return kThreads; }

int solver_max_grid(int tpr, int mt, int num_sms) {
  int nb = 0;
#define MMD_Q(T, M) \
  if (tpr == T && mt == M) nb = max_blocks_for<T, M>();
  MMD_Q(4, 1) MMD_Q(8, 1) MMD_Q(32, 1) MMD_Q(4, 8) MMD_Q(8, 8) MMD_Q(32, 8)
#undef MMD_Q
  nb = nb < 2 ? nb : 2;
  int g = nb * num_sms;
  return g > kThreads ? kThreads : g;
}

cudaError_t launch_solver(const SolverArgs& a, int tpr, int mt, int grid, cudaStream_t st) {
#define MMD_L(T, M) \
  if (tpr == T && mt == M) return launch_tpl<T, M>(a, grid, st);
  MMD_L(4, 1) MMD_L(8, 1) MMD_L(32, 1) MMD_L(4, 8) MMD_L(8, 8) MMD_L(32, 8)
#undef MMD_L
  return cudaErrorInvalidValue;
}

}  // namespace mmd
