// The local solves of the decomposition build on the GPU: psi_j for every
// patch j of a level (Section 2.2's energy-minimising basis restricted to the
// support Omega_j, the patch and whole neighbouring patches).  psi_j
// minimises psi^T A psi subject to phi_i^T psi = delta_ij for the patches i
// inside Omega_j; with L L^T = A[Omega_j, Omega_j], Y = A^{-1} C^T (C the
// constraint rows: phi_i on patch i's rows) and S = C Y,
//   psi_j = Y S^{-1} e_j.
// The patches are independent ("embarrassingly parallel", Appendix A): one
// block per patch at a time, blocks taking patches from an atomic counter.
// Integer inputs (supports, constraint lists) come from the host build, so the
// indexing is the host's; only the floating-point work runs here.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "build_gpu.h"

namespace mmd {

namespace {

constexpr int kThreads = 256;

struct PsiArgs {
  const int32_t* rowptr;   // current level A (natural order)
  const int32_t* col;
  const double* val;
  const double* phi_row;   // phi value of every fine row
  const int32_t* optr;     // np + 1
  const int32_t* orows;    // support rows, ascending per patch
  const int32_t* xidx;     // per support row: its constraint index within the patch's list
  const int32_t* cptr;     // np + 1: constraint list offsets
  const int32_t* jpos;     // np: position of patch j in its own constraint list
  int64_t np;
  int mmax, cmax;          // largest support and constraint list
  double* scratch;         // per block: mmax^2 (L) + cmax * mmax (Y) + cmax^2 (S) + cmax (e)
  double* psival;          // output, aligned with orows
  int* next;               // patch counter (zeroed)
  int* fail;               // set when a local matrix is not positive definite
};

// In-place lower Cholesky of the n x n row-major matrix a (leading dimension
// ld) by the block: right-looking, column by column.  Returns false (all
// threads) if a pivot is not positive.
__device__ bool block_cholesky(double* a, int n, int ld) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x == 0) {
      const double p = a[size_t(c) * ld + c];
      if (!(p > 0.0)) s_bad = 1;
      a[size_t(c) * ld + c] = sqrt(p > 0.0 ? p : 1.0);
    }
    __syncthreads();
    if (s_bad) return false;
    const double dc = a[size_t(c) * ld + c];
    for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) a[size_t(i) * ld + c] /= dc;
    __syncthreads();
    // trailing update of the lower triangle: a warp per row, its lanes on
    // consecutive columns (contiguous in the row-major storage)
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = c + 1 + (threadIdx.x >> 5); i < n; i += nw) {
      const double aic = a[size_t(i) * ld + c];
      for (int k = c + 1 + lane; k <= i; k += 32) a[size_t(i) * ld + k] -= aic * a[size_t(k) * ld + c];
    }
    __syncthreads();
  }
  return true;
}

// L L^T y = b in place for the row b (length n) by one warp: forward then
// backward substitution, each step's dot product shared by the lanes.
__device__ void warp_chol_solve(const double* L, int n, int ld, double* b) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int k = lane; k < i; k += 32) t += L[size_t(i) * ld + k] * b[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) b[i] = (b[i] - t) / L[size_t(i) * ld + i];
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = 0.0;
    for (int k = i + 1 + lane; k < n; k += 32) t += L[size_t(k) * ld + i] * b[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) b[i] = (b[i] - t) / L[size_t(i) * ld + i];
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kThreads) psi_kernel(PsiArgs q) {
  __shared__ int s_j, s_stop;
  const size_t per = size_t(q.mmax) * q.mmax + size_t(q.cmax) * q.mmax + size_t(q.cmax) * q.cmax + q.cmax;
  double* const L = q.scratch + per * blockIdx.x;
  double* const Y = L + size_t(q.mmax) * q.mmax;
  double* const S = Y + size_t(q.cmax) * q.mmax;
  double* const ev = S + size_t(q.cmax) * q.cmax;
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      s_j = atomicAdd(q.next, 1);
      s_stop = (s_j >= q.np) || *(volatile int*)q.fail;
    }
    __syncthreads();
    const int64_t j = s_j;
    const int stop = s_stop;
    __syncthreads();
    if (stop) return;
    const int a = q.optr[j], m = q.optr[j + 1] - a;
    const int c0 = q.cptr[j], nc = q.cptr[j + 1] - c0;
    const int32_t* O = q.orows + a;
    // L = A[O, O]
    for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += blockDim.x) L[t] = 0.0;
    __syncthreads();
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
      const int r = O[x];
      for (int32_t k = q.rowptr[r]; k < q.rowptr[r + 1]; ++k) {
        const int32_t cc = q.col[k];
        int lo = 0, hi = m;  // lower bound of cc in O
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (O[mid] < cc) lo = mid + 1;
          else hi = mid;
        }
        if (lo < m && O[lo] == cc) L[size_t(x) * m + lo] = q.val[k];
      }
    }
    // constraint rows: Y row ai = phi on the rows of constraint patch ai
    for (int64_t t = threadIdx.x; t < int64_t(nc) * m; t += blockDim.x) {
      const int ai = int(t / m), x = int(t % m);
      Y[t] = (q.xidx[a + x] == ai) ? q.phi_row[O[x]] : 0.0;
    }
    __syncthreads();
    if (!block_cholesky(L, m, m)) {
      if (threadIdx.x == 0) atomicExch(q.fail, 1);
      return;
    }
    // Y <- A^{-1} C^T (row ai = column ai), one warp per constraint
    for (int ai = w; ai < nc; ai += nw) warp_chol_solve(L, m, m, Y + size_t(ai) * m);
    __syncthreads();
    // S = C Y, symmetrised; C row ai is nonzero on patch ai's rows only
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
      const int ai = t / nc, bi = t % nc;
      double s = 0.0;
      for (int x = 0; x < m; ++x)
        if (q.xidx[a + x] == ai) s += q.phi_row[O[x]] * Y[size_t(bi) * m + x];
      S[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
      const int ai = t / nc, bi = t % nc;
      if (bi < ai) {
        const double v = 0.5 * (S[size_t(ai) * nc + bi] + S[size_t(bi) * nc + ai]);
        S[size_t(ai) * nc + bi] = v;
        S[size_t(bi) * nc + ai] = v;
      }
    }
    __syncthreads();
    if (!block_cholesky(S, nc, nc)) {
      if (threadIdx.x == 0) atomicExch(q.fail, 1);
      return;
    }
    if (w == 0) {
      for (int t = threadIdx.x; t < nc; t += 32) ev[t] = (t == q.jpos[j]) ? 1.0 : 0.0;
      __syncwarp();
      warp_chol_solve(S, nc, nc, ev);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
      double t = 0.0;
      for (int ai = 0; ai < nc; ++ai) t += Y[size_t(ai) * m + x] * ev[ai];
      q.psival[a + x] = t;
    }
    __syncthreads();
  }
}

template <typename T>
int up(T** d, const std::vector<T>& h) {
  if (cudaMalloc(d, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) return -1;
  if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return -1;
  return 0;
}

}  // namespace

int psi_solves_gpu(const HCSR& A, const std::vector<int32_t>& patch_of, const std::vector<double>& phi_of_row,
                   const std::vector<int32_t>& optr, const std::vector<int32_t>& orows, int64_t np,
                   std::vector<double>& psival, std::string& err) {
  // constraint lists (patches inside each support, ascending id) and every
  // support row's index in its patch's list -- integer work, as on the host
  std::vector<int32_t> cptr(np + 1, 0), cpat, xidx(orows.size()), jpos(np);
  int mmax = 1, cmax = 1;
  for (int64_t j = 0; j < np; ++j) {
    const int a = optr[j], m = optr[j + 1] - a;
    std::vector<int32_t> up_(m);
    for (int x = 0; x < m; ++x) up_[x] = patch_of[orows[a + x]];
    std::sort(up_.begin(), up_.end());
    up_.erase(std::unique(up_.begin(), up_.end()), up_.end());
    for (int x = 0; x < m; ++x)
      xidx[a + x] = int32_t(std::lower_bound(up_.begin(), up_.end(), patch_of[orows[a + x]]) - up_.begin());
    jpos[j] = int32_t(std::lower_bound(up_.begin(), up_.end(), (int32_t)j) - up_.begin());
    cptr[j + 1] = cptr[j] + (int32_t)up_.size();
    cpat.insert(cpat.end(), up_.begin(), up_.end());
    mmax = std::max(mmax, m);
    cmax = std::max(cmax, (int)up_.size());
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max<int64_t>(1, std::min<int64_t>(int64_t(nsm) * 4, np));
  const size_t per = size_t(mmax) * mmax + size_t(cmax) * mmax + size_t(cmax) * cmax + cmax;
  PsiArgs q{};
  int32_t *rp = nullptr, *ci = nullptr, *op = nullptr, *orr = nullptr, *xi = nullptr, *cp = nullptr, *jp = nullptr;
  double *va = nullptr, *ph = nullptr, *scr = nullptr, *out = nullptr;
  int* ctr = nullptr;
  int rc = 0;
  if (up(&rp, A.rowptr) || up(&ci, A.col) || up(&va, A.val) || up(&ph, phi_of_row) || up(&op, optr) ||
      up(&orr, orows) || up(&xi, xidx) || up(&cp, cptr) || up(&jp, jpos) ||
      cudaMalloc(&scr, per * grid * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&out, std::max<size_t>(orows.size(), 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctr, 2 * sizeof(int)) != cudaSuccess) {
    err = "device allocation for the local psi solves failed";
    rc = -1;
  }
  if (!rc) {
    cudaMemset(ctr, 0, 2 * sizeof(int));
    q.rowptr = rp;
    q.col = ci;
    q.val = va;
    q.phi_row = ph;
    q.optr = op;
    q.orows = orr;
    q.xidx = xi;
    q.cptr = cp;
    q.jpos = jp;
    q.np = np;
    q.mmax = mmax;
    q.cmax = cmax;
    q.scratch = scr;
    q.psival = out;
    q.next = ctr;
    q.fail = ctr + 1;
    psi_kernel<<<grid, kThreads>>>(q);
    int fail = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&fail, ctr + 1, sizeof(int), cudaMemcpyDeviceToHost) !=
                                                 cudaSuccess) {
      err = "the local psi solve kernel failed";
      rc = -1;
    } else if (fail) {
      err = "a neighbourhood matrix is not positive definite";
      rc = 1;
    } else {
      psival.resize(orows.size());
      if (!orows.empty() &&
          cudaMemcpy(psival.data(), out, orows.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        err = "copy of the psi values failed";
        rc = -1;
      }
    }
  }
  cudaFree(rp);
  cudaFree(ci);
  cudaFree(va);
  cudaFree(ph);
  cudaFree(op);
  cudaFree(orr);
  cudaFree(xi);
  cudaFree(cp);
  cudaFree(jp);
  cudaFree(scr);
  cudaFree(out);
  cudaFree(ctr);
  return rc;
}

}  // namespace mmd
