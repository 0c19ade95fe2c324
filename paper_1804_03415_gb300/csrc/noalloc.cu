// mmd_cg_solve_noalloc: conjugate gradients on a caller's device CSR matrix
// with every byte of working memory taken from one fixed array compiled into
// the library, so the call itself never allocates.
//
// Who needs this: code that may not call cudaMalloc at the moment it wants a
// solve -- a service that reserves all device memory up front and treats any
// later allocation as a failure, a real-time loop that cannot afford the
// device-wide synchronisation an allocation can cause, or a host framework
// that hands the library only its inputs and outputs.  Such callers still
// pass b and x; the vectors r, p, q, the reduction partials and the grid
// barrier counter live in g_noalloc_scratch below.
//
// The array is a file-scope __device__ variable: each GPU that loads the
// library holds its own copy (about 8 MB) until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on each
// device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; that first call should therefore come
// before any stream capture.  Every call shares the same array and it keeps
// the previous call's contents, so each call clears what must start at zero
// (the barrier counter and the status word) with a memset on its stream
// before the kernel, and two calls that overlap on the GPU (different
// streams, no ordering) would race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/mmdeig.h"
#include "dev_common.cuh"
#include "mmd_internal.h"

namespace mmd {
namespace {

constexpr int64_t kMaxN = MMD_NOALLOC_MAX_N;
constexpr int kThreadsNA = 512;
constexpr int kMaxBlocks = 1024;
// layout (doubles): r[kMaxN] p[kMaxN] q[kMaxN] partials[2 * kMaxBlocks] control[64]
constexpr int64_t kOffR = 0, kOffP = kMaxN, kOffQ = 2 * kMaxN, kOffPart = 3 * kMaxN;
constexpr int64_t kOffCtl = 3 * kMaxN + 2 * kMaxBlocks;
constexpr int64_t kScratchDoubles = kOffCtl + 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct NAArgs {
  int64_t n;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const double* b;
  double* x;
  double tol;
  int maxit;
  double* scratch;  // device address of g_noalloc_scratch
  GridBarrier bar;
};

__device__ double na_block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// partial of slot s -> every block reads all partials in the same order
__device__ double na_reduce(const double* part, int slot) {
  double t = 0.0;
  for (int i = 0; i < (int)gridDim.x; ++i) t += part[slot * kMaxBlocks + i];
  return t;
}

// Plain CG (Hestenes-Stiefel), x0 = 0, relative residual ||r|| <= tol ||b||.
// Thread per row; dot products fused into the SpMV and the updates.
__global__ void __launch_bounds__(kThreadsNA) na_cg_kernel(NAArgs a) {
  __shared__ double red[32];
  grid_sync_init();
  double* r = a.scratch + kOffR;
  double* p = a.scratch + kOffP;
  double* q = a.scratch + kOffQ;
  double* part = a.scratch + kOffPart;
  double* ctl = a.scratch + kOffCtl;  // ctl[0] = iterations, ctl[1] = converged
  const int64_t n = a.n;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nthr = int64_t(gridDim.x) * blockDim.x;
  double acc = 0.0;
  for (int64_t i = tid; i < n; i += nthr) {
    const double bv = a.b[i];
    a.x[i] = 0.0;
    r[i] = bv;
    p[i] = bv;
    acc = fma(bv, bv, acc);
  }
  acc = na_block_sum(acc, red);
  if (threadIdx.x == 0) part[0 * kMaxBlocks + blockIdx.x] = acc;
  if (!grid_sync(a.bar)) return;
  const double bb = na_reduce(part, 0);
  double rr = bb;
  const double stop = a.tol * a.tol * bb;
  int it = 0;
  bool conv = !(rr > stop);
  while (!conv && it < a.maxit) {
    ++it;
    acc = 0.0;
    for (int64_t i = tid; i < n; i += nthr) {
      double s = 0.0;
      for (int32_t k = a.rp[i]; k < a.rp[i + 1]; ++k) s = fma(a.va[k], p[a.ci[k]], s);
      q[i] = s;
      acc = fma(p[i], s, acc);
    }
    acc = na_block_sum(acc, red);
    if (threadIdx.x == 0) part[1 * kMaxBlocks + blockIdx.x] = acc;
    if (!grid_sync(a.bar)) return;
    const double pq = na_reduce(part, 1);
    if (!(pq > 0.0)) {
      if (tid == 0) atomicExch(a.bar.status, (int)DEV_NOTSPD);
      break;
    }
    const double alpha = rr / pq;
    acc = 0.0;
    for (int64_t i = tid; i < n; i += nthr) {
      a.x[i] = fma(alpha, p[i], a.x[i]);
      const double rv = fma(-alpha, q[i], r[i]);
      r[i] = rv;
      acc = fma(rv, rv, acc);
    }
    acc = na_block_sum(acc, red);
    if (threadIdx.x == 0) part[0 * kMaxBlocks + blockIdx.x] = acc;
    if (!grid_sync(a.bar)) return;
    const double rn = na_reduce(part, 0);
    conv = !(rn > stop);
    const double beta = rn / rr;
    rr = rn;
    if (!conv)
      for (int64_t i = tid; i < n; i += nthr) p[i] = fma(beta, p[i], r[i]);
    if (!grid_sync(a.bar)) return;
  }
  if (tid == 0) {
    ctl[0] = (double)it;
    ctl[1] = conv ? 1.0 : 0.0;
  }
}

double* g_scratch_addr[64] = {nullptr};
int g_max_grid[64] = {0};
std::mutex g_setup_mu;  // serialises the per-device set-up of host threads' first calls

}  // namespace
}  // namespace mmd

using namespace mmd;

extern "C" int mmd_cg_solve_noalloc(const mmd_csr* A, const double* b, double* x, double tol, int max_iter,
                                    int64_t* iters, void* stream) {
  if (!A || !b || !x || !A->on_device || A->n < 1 || !(tol > 0) || max_iter < 1) {
    set_error("mmd_cg_solve_noalloc: needs a device CSR (on_device = 1), device b and x, tol > 0, max_iter >= 1");
    return MMD_EINVAL;
  }
  if (A->n > kMaxN) {
    set_error("mmd_cg_solve_noalloc: n = " + std::to_string(A->n) + " exceeds the fixed scratch limit of " +
              std::to_string((long long)kMaxN) + " rows (MMD_NOALLOC_MAX_N)");
    return MMD_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("mmd_cg_solve_noalloc: no usable current CUDA device");
    return MMD_ECUDA;
  }
  std::unique_lock<std::mutex> setup_lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {  // once per device, with that device current
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("mmd_cg_solve_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return MMD_ECUDA;
    }
    int nsm = 0, nb = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, na_cg_kernel, kThreadsNA, 0);
    int g = nb * nsm;
    if (g > kMaxBlocks) g = kMaxBlocks;
    if (g < 1) {
      set_error("mmd_cg_solve_noalloc: kernel cannot be made resident");
      return MMD_ECUDA;
    }
    g_max_grid[dev] = g;
    g_scratch_addr[dev] = (double*)ptr;
  }
  double* scr = g_scratch_addr[dev];
  const int max_grid = g_max_grid[dev];
  setup_lock.unlock();
  cudaStream_t st = (cudaStream_t)stream;
  NAArgs a;
  a.n = A->n;
  a.rp = A->rowptr;
  a.ci = A->col;
  a.va = A->val;
  a.b = b;
  a.x = x;
  a.tol = tol;
  a.maxit = max_iter;
  a.scratch = scr;
  a.bar.count = (unsigned*)(scr + kOffCtl + 8);
  a.bar.gen = (unsigned*)(scr + kOffCtl + 24);
  a.bar.status = (int*)(scr + kOffCtl + 40);
  a.bar.timeout_ns = 2000000000LL;
  // the array keeps the previous call's contents: zero the control block
  if (cudaMemsetAsync(scr + kOffCtl, 0, 64 * sizeof(double), st) != cudaSuccess) {
    set_error("mmd_cg_solve_noalloc: clearing the control words failed");
    return MMD_ECUDA;
  }
  int64_t rows_per_block = (A->n + kThreadsNA - 1) / kThreadsNA;
  int grid = (int)(rows_per_block < max_grid ? rows_per_block : max_grid);
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)na_cg_kernel, dim3(grid), dim3(kThreadsNA), args, 0, st);
  if (e != cudaSuccess) {
    set_error(std::string("mmd_cg_solve_noalloc: launch failed: ") + cudaGetErrorString(e));
    return MMD_ECUDA;
  }
  double ctl[2] = {0, 0};
  int status = 0;
  if (cudaMemcpyAsync(ctl, scr + kOffCtl, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&status, a.bar.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("mmd_cg_solve_noalloc: reading the result failed");
    return MMD_ECUDA;
  }
  if (iters) *iters = (int64_t)ctl[0];
  if (status == DEV_TIMEOUT) {
    set_error("mmd_cg_solve_noalloc: a grid barrier wait exceeded its time limit");
    return MMD_ETIMEOUT;
  }
  if (status == DEV_NOTSPD) {
    set_error("mmd_cg_solve_noalloc: p^T A p <= 0 (matrix not SPD)");
    return MMD_ENOTSPD;
  }
  if (ctl[1] != 1.0) {
    set_error("mmd_cg_solve_noalloc: max_iter reached");
    return MMD_ENOCONV;
  }
  return MMD_OK;
}
