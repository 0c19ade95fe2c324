// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mmd {

// Status word written by kernels (0 = fine).
enum DevStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BREAKDOWN = 2, DEV_NOTSPD = 3, DEV_NOCONV = 4 };

struct GridBarrier {
  unsigned int* count;  // monotone arrival counter (zeroed before each launch)
  unsigned int* gen;    // unused (kept for layout)
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

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Phase counter of the grid barrier, one per block.
__shared__ unsigned g_bar_phase;

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// The counter only grows: phase t of the launch is complete when it reaches
// t * gridDim.  One release-add per block, then an acquire poll with a short
// sleep between polls (the counter lives on its own 128-byte line).  A wait
// gives up after timeout_ns: the status word is set and every block that
// sees it returns false (callers leave the kernel), so the launch ends in
// bounded time.  The counter is zeroed before every launch and
// grid_sync_init() must run at kernel entry.
__device__ __forceinline__ void grid_sync_init() {
  if (threadIdx.x == 0) g_bar_phase = 0;
  __syncthreads();
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned target = (++g_bar_phase) * nb;
    __threadfence();
    red_release_add(b.count, 1u);
    int ok = 1;
    const long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire(b.count) < target) {
      __nanosleep(20);
      if (((++spins) & 255u) == 1u) {  // first poll, then every 256th
        // another block's status (not SPD, a timeout) ends the wait as it is;
        // our own time limit turns an OK status into a timeout
        if (ld_acquire_int(b.status) != DEV_OK) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > b.timeout_ns) {
          atomicCAS(b.status, (int)DEV_OK, (int)DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
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
