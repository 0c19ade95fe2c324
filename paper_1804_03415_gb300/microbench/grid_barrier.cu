// Cost of the solver's grid barrier (dev_common.cuh: monotone counter, bounded
// wait) on cooperative grids of 16..all SMs x 1024 threads, 20,000 barriers:
// mode 0 = barrier alone, mode 1 = a reduction round of the kind the CG
// kernel runs (FP64 block sum by shuffle trees, partial written, barrier, one
// warp reads and sums all blocks' partials).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o grid_barrier grid_barrier.cu && ./grid_barrier
#include <cstdio>
#include <cuda_runtime.h>
#include "../csrc/dev_common.cuh"
using namespace mmd;
__global__ void k_bar(GridBarrier b, int K, double* part, double* out, int mode) {
  grid_sync_init();
  __shared__ double red[32];
  double acc = threadIdx.x * 1e-3;
  for (int k = 0; k < K; ++k) {
    if (mode == 1) {  // block FP64 sum + write partial + barrier + warp reads all partials
      double t = block_sum(acc, red);
      if (threadIdx.x == 0) part[(k & 1) * 1024 + blockIdx.x] = t;
    }
    if (!grid_sync(b)) return;
    if (mode == 1) {
      if (threadIdx.x < 32) {
        double t = 0; for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) t += part[(k & 1) * 1024 + i];
        t = warp_sum(t); if (threadIdx.x == 0) red[0] = t;
      }
      __syncthreads();
      acc += red[0] * 1e-30;
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = acc;
}
int main() {
  unsigned* cnt; int* st; double* part; double* out;
  cudaMalloc(&cnt, 256); cudaMalloc(&st, 256); cudaMalloc(&part, 2048 * 8); cudaMalloc(&out, 8);
  int nsm; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  int grids[] = {16, 38, 76, nsm};
  for (int mode = 0; mode < 2; ++mode)
    for (int g : grids) {
      GridBarrier b{cnt, cnt + 32, st, 2000000000LL};
      int K = 20000;
      for (int rep = 0; rep < 2; ++rep) {
        cudaMemset(cnt, 0, 256); cudaMemset(st, 0, 256);
        cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
        void* args[] = {&b, &K, &part, &out, &mode};
        cudaEventRecord(e0);
        cudaError_t e = cudaLaunchCooperativeKernel((void*)k_bar, dim3(g), dim3(1024), args, 0, 0);
        cudaEventRecord(e1); cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        int hs; cudaMemcpy(&hs, st, 4, cudaMemcpyDeviceToHost);
        if (rep) printf("mode %d grid %3d: %.3f us per barrier (status %d, %s)\n", mode, g, ms * 1e3 / K, hs, cudaGetErrorString(e));
      }
    }
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
