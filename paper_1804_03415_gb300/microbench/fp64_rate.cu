// FP64 (and FP32) FMA issue rate on one SM of the GPU: 1..32 warps run
// chains of FMAs (1, 4 or 8 independent accumulators per thread), each warp
// times its chain with clock64.  Prints cycles per warp-instruction and FMAs
// per clock for the SM.  The solver's design (few FP64 instructions, spread
// over the SM's four sub-partitions) rests on these numbers.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_rate fp64_rate.cu && ./fp64_rate
#include <cstdio>
#include <cuda_runtime.h>

__global__ void k_fma(int iters, int ilp, double* out, long long* cyc) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  const double m = 0.999999, c = 1e-7;
  __syncthreads();
  long long t0 = clock64();
  if (ilp == 1) {
    for (int i = 0; i < iters; ++i) a0 = fma(a0, m, c);
  } else if (ilp == 4) {
    for (int i = 0; i < iters; i += 4) {
      a0 = fma(a0, m, c);
      a1 = fma(a1, m, c);
      a2 = fma(a2, m, c);
      a3 = fma(a3, m, c);
    }
  } else {
    for (int i = 0; i < iters; i += 8) {
      a0 = fma(a0, m, c);
      a1 = fma(a1, m, c);
      a2 = fma(a2, m, c);
      a3 = fma(a3, m, c);
      a4 = fma(a4, m, c);
      a5 = fma(a5, m, c);
      a6 = fma(a6, m, c);
      a7 = fma(a7, m, c);
    }
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if ((threadIdx.x & 31) == 0) cyc[blockIdx.x * 32 + (threadIdx.x >> 5)] = t1 - t0;
}

__global__ void k_ffma(int iters, float* out, long long* cyc) {
  float a0 = threadIdx.x * 1e-3f, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  const float m = 0.999f, c = 1e-4f;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < iters; i += 4) {
    a0 = fmaf(a0, m, c);
    a1 = fmaf(a1, m, c);
    a2 = fmaf(a2, m, c);
    a3 = fmaf(a3, m, c);
  }
  long long t1 = clock64();
  out[threadIdx.x] = a0 + a1 + a2 + a3;
  if ((threadIdx.x & 31) == 0) cyc[threadIdx.x >> 5] = t1 - t0;
}

int main() {
  double* out;
  long long* cyc;
  float* outf;
  cudaMalloc(&out, 1024 * 8 * 4);
  cudaMalloc(&cyc, 32 * 8 * 4);
  cudaMalloc(&outf, 1024 * 4);
  long long h[32];
  const int iters = 4096;
  const int ws[] = {1, 2, 4, 8, 16, 32};
  const int ilps[] = {1, 4, 8};
  for (int il : ilps)
    for (int w : ws) {
      k_fma<<<1, w * 32>>>(iters, il, out, cyc);
      k_fma<<<1, w * 32>>>(iters, il, out, cyc);
      cudaMemcpy(h, cyc, 8 * w, cudaMemcpyDeviceToHost);
      long long mx = 0;
      for (int i = 0; i < w; ++i) mx = h[i] > mx ? h[i] : mx;
      printf("dfma ilp=%d warps=%2d cycles/warp-instr=%.2f  SM fma/clk=%.3f\n", il, w, (double)mx / iters,
             (double)w * 32 * iters / mx);
    }
  for (int w : ws) {
    k_ffma<<<1, w * 32>>>(iters, outf, cyc);
    k_ffma<<<1, w * 32>>>(iters, outf, cyc);
    cudaMemcpy(h, cyc, 8 * w, cudaMemcpyDeviceToHost);
    long long mx = 0;
    for (int i = 0; i < w; ++i) mx = h[i] > mx ? h[i] : mx;
    printf("ffma ilp=4 warps=%2d cycles/warp-instr=%.2f  SM fma/clk=%.3f\n", w, (double)mx / iters,
           (double)w * 32 * iters / mx);
  }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
