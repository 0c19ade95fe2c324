// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mmd {

// Status word written by kernels (0 = fine).
enum DevStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BREAKDOWN = 2, DEV_NOTSPD = 3 };

struct GridBarrier {
  unsigned int* count;  // arrivals in the current phase
  unsigned int* gen;    // phase counter
  int* status;          // set to DEV_TIMEOUT when a wait gives up
  long long timeout_ns; // limit of one wait
};

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_int(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// last block to arrive resets the count and advances the phase; the others
// wait for the phase to change, for at most timeout_ns.  On timeout the
// status word is set; the function then returns false on every block that
// sees the status (callers leave the kernel).  Returns true when all blocks
// passed.
__device__ __forceinline__ bool grid_sync(const GridBarrier& b) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire(b.gen);
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned arrived = atomicAdd(b.count, 1u);
    int ok = 1;
    if (arrived == nb - 1) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      const long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire(b.gen) == g) {
        if (((++spins) & 63u) == 0u) {
          if (ld_acquire_int(b.status) != DEV_OK || global_ns() - t0 > b.timeout_ns) {
            atomicExch(b.status, (int)DEV_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    if (ok && ld_acquire_int(b.status) != DEV_OK) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) { return group_sum<32>(v); }

// Sum of v over the block (fixed tree order); result valid in every thread.
// red: shared scratch of >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

}  // namespace mmd
