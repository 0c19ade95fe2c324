// Device-side eigensolver driver (internal).
#pragma once

#include <cuda_runtime.h>

#include "mmd_internal.h"

namespace mmd {

int level_spmv(mmd_handle* h, int k, int which, const double* x, double* y, cudaStream_t st);
int level_op(mmd_handle* h, int k, const double* x, double* y, double tol, int max_iter, int64_t* iters,
             cudaStream_t st);
int level_bsolve(mmd_handle* h, int k, const double* q, double* x, double tol, int max_iter, int64_t* iters,
                 cudaStream_t st);
int run_eig(mmd_handle* h, int N, double tol, const mmd_eig_opts& o, double* lambda, double* V, int outdev,
            mmd_eig_stats* stats);
void free_workspace(mmd_handle* h);

extern int64_t g_kernel_launches;
void set_tri_scratch(double* bounds, double* e2, int* cstart, int* ncl, double* work, int* iwork);

}  // namespace mmd
