// Device-side eigensolver driver (internal).
#pragma once

#include <cuda_runtime.h>

#include "mmd_internal.h"

namespace mmd {

int level_spmv(mmd_handle* h, int k, int which, const double* x, double* y, cudaStream_t st);
int level_spmv_timed(mmd_handle* h, int k, int which, const double* x, double* y, int reps, float* ms,
                     cudaStream_t st);
int level_op(mmd_handle* h, int k, const double* x, double* y, double tol, int max_iter, int64_t* iters,
             cudaStream_t st);
int level_op_block(mmd_handle* h, int k, int m, const double* x, double* y, double tol, int max_iter,
                   int64_t* iters, int precision, cudaStream_t st);
int level_bsolve(mmd_handle* h, int k, const double* q, double* x, double tol, int max_iter, int64_t* iters,
                 cudaStream_t st);
int level_vcycle(mmd_handle* h, int m, const double* R, double* Z, int deg, cudaStream_t st);
// Candidate grids of the solver autotuner (blocks of 1024 threads, one per SM)
constexpr int kTuneGrids[8] = {2, 4, 8, 16, 32, 64, 96, 152};
int tune_solver(mmd_handle* h);
int level_poly(mmd_handle* h, int m, const double* R, double* Z, int deg, double ratio, cudaStream_t st);
int run_eig(mmd_handle* h, int N, double tol, const mmd_eig_opts& o, double* lambda, double* V, int outdev,
            mmd_eig_stats* stats);
int run_grad(mmd_handle* h, const double* gl, const double* Gv, int in_dev, double* out, int out_dev,
             const mmd_eig_opts& o);
void free_workspace(mmd_handle* h);

void set_tri_scratch(double* bounds, double* e2, int* cstart, int* ncl, double* work, int* iwork);

}  // namespace mmd
