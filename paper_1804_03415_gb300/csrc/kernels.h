// Launch wrappers of the library's CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dev_common.cuh"

namespace mmd {

// SELL-32 view of a sparse matrix (see DCSR).
struct Sell {
  int64_t nrows = 0;
  int64_t nslices = 0;
  const int32_t* ptr = nullptr;
  const int32_t* len = nullptr;
  const int32_t* row = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const float* val32 = nullptr;
  const float2* val2 = nullptr;  // double-float copy: value = hi + lo
  int variant = -1;  // single-column SpMV kernel picked by k_spmv_autotune (-1: not tuned)
};

// One level of the V-cycle preconditioner (FP32 work, device order of the
// level): A^(k), Psi^(k+1) and its transpose, 1 / diag A^(k), the Gershgorin
// bound of D^{-1} A^(k), and MT-interleaved work vectors.
// CSR view (device order, FP32 values) of a V-cycle matrix whose rows are
// long enough to share a row among g lanes (g = 0: use the SELL copy).
struct Csr32 {
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const float* val = nullptr;
  int64_t nrows = 0;
  int g = 0;
};

struct MGLevel {
  Sell A;               // A^(k) (val32 used)
  Sell P;               // Psi^(k+1): rows of level k, columns of level k + 1
  Sell PT;              // Psi^(k+1)^T: rows of level k + 1, columns of level k
  Csr32 cA, cP, cPT;    // the same matrices as CSR, used when their g > 0
  const float* dinv;    // n
  double hi;            // upper end of the Chebyshev interval
  // Chebyshev step st (pre- and post-smoothing alike): d = c1[st] d + c2[st] D^{-1} (r - A x), x += d
  float c1[8], c2[8];
  int64_t n;            // N^(k)
  float *r, *x, *x2, *d;  // n x MT each: right-hand side, iterate (ping-pong), direction / residual
};

// Polynomial preconditioner of the level-0 solves (mode 4, FP32 work):
// z = p(D^{-1} A) D^{-1} r, deg steps of the Chebyshev iteration for A z = r
// from z = 0 on the interval [hi / ratio, hi] of D^{-1} A (hi its Gershgorin
// bound); step st: d = c1[st] d + c2[st] D^{-1} (r - A x), x += d (c1[0] = 0).
struct PolyPrec {
  int deg;
  float c1[32], c2[32];
  const float* dinv;      // n
  Csr32 cA;               // CSR view of A (g > 0: rows shared by g lanes)
  float *r, *x, *x2, *d;  // n x MT each, interleaved
};

struct SolverArgs {
  int mode;  // 0 CG, 1 flexible PCG with inner CG on M, 2 CG on P A P, 3 flexible PCG with the V-cycle,
             // 4 flexible PCG with the Chebyshev polynomial preconditioner
  int64_t n;
  Sell A;
  Sell M;
  const int32_t* seg_ptr;
  const double* phi;
  int64_t nseg;
  int m;
  int64_t ld;
  const void* b;   // T = double, or float when fp32 = 1
  void* x;
  int x0;
  void *r, *p, *q, *z;
  void *ir, *ip, *iq;
  int fp32;        // 1: FP32 instance (matrix val32, FP32 vectors)
  int df;          // 1: double-float CG (mode 0): matrix val2, vectors as FP32 pairs, FP64 b and x
  // mode 0 with fp32 = 1 and b64 != NULL: FP32 CG with FP64 reliable updates;
  // b64 / x64 (n x m, ld) are the FP64 right-hand side and solution
  const double* b64;
  double* x64;
  double tol, itol;
  int maxit, imaxit;
  double* red;         // [4][MT][grid]
  int64_t* it_out;     // [m]
  int64_t* in_out;     // [1], accumulated
  int* conv;           // [m]
  GridBarrier bar;
  // mode 3: the V-cycle (levels 0 .. mg_K - 1 in device memory, dense coarsest inverse)
  const MGLevel* mg;
  int mg_K, mg_deg;
  const float* mg_kinv;  // nK x nK, column-major
  float *mg_rK, *mg_xK;  // nK x MT
  int64_t mg_nK;
  int mg_only;  // 1: apply z = V(b) once (x = z, column-major) instead of solving
  PolyPrec poly;  // mode 4
};

// Many right-hand sides of one level-0 solve (CG on A, the refinement's
// block) in one persistent launch, double-float arithmetic (wide.cu).
constexpr int kWideMaxCols = 128;
struct WideArgs {
  int64_t n;
  int m;                    // columns, 1 .. kWideMaxCols
  int64_t ld;               // leading dimension of b and x
  const int32_t* rowptr;    // A (CSR, device order)
  const int32_t* col;
  const float2* val2;       // values as FP32 pairs
  const double* val;        // values in FP64 (the residual check)
  const double* b;          // n x m column-major, FP64
  double* x;                // n x m column-major, FP64 (x0 on entry when x0)
  int x0;
  void *r, *p, *s, *w, *xd; // n x m row-major pairs (8 bytes each)
  double* q64;              // n x m row-major FP64
  void* red;                // [2][m][grid] float2 partials
  double* red64;            // [2][m][grid] FP64 partials
  double tol;
  int maxit;
  int64_t* it_out;          // m
  int* conv;                // m
  GridBarrier bar;
};
int wide_max_grid(int num_sms);
cudaError_t launch_wide_cg(const WideArgs& a, int grid, cudaStream_t st);

int solver_threads(int mt);
int solver_max_grid(int mt, int num_sms);
cudaError_t launch_solver(const SolverArgs& a, int mt, int grid, cudaStream_t st);

// ---- vector / sparse kernels (blas.cu)
void k_fill(double* x, int64_t n, double v, cudaStream_t st);
void k_copy(double* y, const double* x, int64_t n, cudaStream_t st);
void k_scal(double* x, int64_t n, double a, cudaStream_t st);
void k_axpy(double* y, const double* x, int64_t n, double a, cudaStream_t st);
// y = A x (SELL-32), columns m of ld (x, y column-major); one column runs the
// single-column variant in A.variant when it has been tuned
void k_spmv(const Sell& A, const double* x, int64_t ldx, double* y, int64_t ldy, int m, cudaStream_t st);
// Times every single-column SpMV variant on A (x, y: scratch vectors of A's
// size) with events on st and returns the fastest one's index; ms_out (may be
// NULL) receives each variant's mean time.  Variants differ in the entries
// in flight per lane, the block size and the register bound.
int k_spmv_autotune(const Sell& A, const double* x, double* y, cudaStream_t st, float* ms_out);
int k_spmv_variants();
// dot products: out[c] = sum_i x(i,c) y(i,c), deterministic two-stage; scratch >= 1024*m doubles
void k_dots(const double* x, const double* y, int64_t n, int64_t ld, int m, double* out, double* scratch,
            cudaStream_t st);
// h = B^T u (B: n x j col-major, ldb) deterministic; scratch >= chunks*j
void k_gemv_t(const double* B, int64_t ldb, int64_t n, int j, const double* u, double* h, double* scratch,
              cudaStream_t st);
// y += alpha * B h  (B: n x j)
void k_gemv_n(const double* B, int64_t ldb, int64_t n, int j, const double* h, double alpha, double* y,
              cudaStream_t st);
// C (m x n, ldc) = alpha A^T B + beta C, A: K x m (lda), B: K x n (ldb); deterministic split-K
void k_gemm_tn(int m, int n, int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, double* scratch, int64_t scratch_len, cudaStream_t st);
// C (M x n, ldc) = alpha A B + beta C, A: M x k (lda), B: k x n (ldb); M long
void k_gemm_nn(int64_t M, int n, int k, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, cudaStream_t st);
// gather / scatter by permutation: y[i] = x[perm[i]] (columns m, ld)
void k_gather(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y, int64_t ldy,
              cudaStream_t st);
void k_scatter(const double* x, int64_t ldx, const int32_t* perm, int64_t n, int m, double* y, int64_t ldy,
               cudaStream_t st);
// project each column onto range(P): x -= phi (phi^T x) per segment
void k_project(double* x, int64_t ld, int m, const int32_t* seg_ptr, const double* phi, int64_t nseg,
               cudaStream_t st);
// G[e] = sum_i U(r_e, i) V(c_e, i) over a CSR pattern (U, V: n x N, ld)
void k_sddmm(const int32_t* rp, const int32_t* ci, int64_t n, const double* U, const double* V, int64_t ld, int N,
             double* G, cudaStream_t st);
// r = b - y (FP64); f = (float) d; x += (double) f  (n x m, ld n)
void k_sub(double* r, const double* b, const double* y, int64_t n, cudaStream_t st);
void k_to_f32(float* f, const double* d, int64_t n, cudaStream_t st);
void k_add_f32(double* x, const float* f, int64_t n, cudaStream_t st);
// columns: x(:,c) *= s[c]
void k_scale_cols(double* x, int64_t ld, int64_t n, int m, const double* s, cudaStream_t st);
// SplitMix64 counter random vector in [-1, 1)
void k_random(double* x, int64_t n, uint64_t seed, uint64_t stream, const int32_t* perm, cudaStream_t st);
// column norms^2: out[c] = sum x(:,c)^2
// sign fix + normalise columns (largest |.| positive, ties lowest index)
void k_normalise_sign(double* V, int64_t ld, int64_t n, int m, double* scratch, cudaStream_t st);
// residual norms ||A v - l v||: out[c]
void k_residuals(const Sell& A, int64_t n, const double* V, int64_t ld, int m, const double* lam, double* out,
                 double* scratch, cudaStream_t st);

// ---- small dense (dense.cu); all matrices column-major
// eigenvalues of symmetric tridiagonal (d: n, e: n-1) by bisection, ascending
void k_tri_eigvals(const double* d, const double* e, int n, double* w, cudaStream_t st);
// implicit-QR eigen-decomposition of a symmetric tridiagonal (n <= 6000):
// w ascending; Z (n x n) full eigenvectors if non-NULL; zl (n) last row of Z if non-NULL
void k_tri_ql(const double* d, const double* e, int n, double* w, double* Z, int ldz, double* zl, int* status,
              cudaStream_t st);
// p explicitly shifted QR steps on tridiagonal (d, e) of order n with shifts sh[0..p-1];
// Q (n x n) is overwritten with the accumulated orthogonal factor (starting from I).
void k_tri_qr_sweeps(double* d, double* e, int n, const double* sh, int p, double* Q, int ldq, cudaStream_t st);
// parallel two-sided Jacobi (cooperative): S (m x m, ld m) -> diagonal (eigenvalues, unsorted),
// V (m x m) eigenvectors; work >= m + 4 doubles, iwork >= 30 ints
cudaError_t k_syev_jacobi(double* S, int m, double* V, double* work, int* iwork, GridBarrier bar, cudaStream_t st);

// Upper bound on the blocks of the calling host thread's cooperative launches
// (0 = none).  Concurrent solves on several streams split the SMs so that
// every cooperative grid stays resident next to the others.
void set_coop_grid_cap(int blocks);
int coop_grid_cap();
// B(:, c) = A(:, perm[c])
void k_permute_cols(const double* A, int lda, int64_t nrows, const int* perm, int ncols, double* B, int ldb,
                    cudaStream_t st);
// Cholesky A = R^T R (upper R in place), status set on failure; Rinv = R^{-1} upper
void k_potrf_upper(double* A, int lda, int n, int* dev_status, cudaStream_t st);
void k_trinv_upper(const double* R, int ldr, int n, double* Rinv, int ldri, cudaStream_t st);
// lower Cholesky L (in place), and C = L^{-1} A L^{-T} for the generalized problem
void k_potrf_lower(double* A, int lda, int n, int* dev_status, cudaStream_t st);
void k_trsm_llnn(const double* L, int ldl, int n, double* B, int ldb, int nrhs, cudaStream_t st);  // B = L^{-1} B
void k_trsm_lltn(const double* L, int ldl, int n, double* B, int ldb, int nrhs, cudaStream_t st);  // B = L^{-T} B
void k_transpose_sq(const double* A, int lda, int n, double* B, int ldb, cudaStream_t st);
void k_symmetrise(double* A, int lda, int n, cudaStream_t st);
void k_csr_to_dense(const int32_t* rp, const int32_t* ci, const double* va, int n, double* D, int ldd,
                    cudaStream_t st);
}  // namespace mmd
