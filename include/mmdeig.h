/*
 * mmdeig.h -- C ABI of a GB300 (sm_103a) implementation of the hierarchically
 * preconditioned eigensolver of Hou, Huang, Lam and Zhang, "A Fast
 * Hierarchically Preconditioned Eigensolver Based on Multiresolution Matrix
 * Decomposition" (arXiv 1804.03415).
 *
 * The library computes the N leftmost eigenpairs of a sparse symmetric
 * positive definite matrix A.  It first builds a Multiresolution Matrix
 * Decomposition (Section 2.3: levels A^(k) = Psi^(k)^T A^(k-1) Psi^(k),
 * M^(k) = Psi^(k)^T M^(k-1) Psi^(k), complement bases U^(k)), then runs the
 * Hierarchical Eigenpair Computation (Algorithm 6): a dense generalized
 * eigenproblem on the coarsest level, then per level an Eigenpair Refinement
 * (Algorithm 5) and an Eigenpair Extension (Algorithm 4, implicitly restarted
 * M-Lanczos, Algorithms 2-3), whose operator is Operator OP: PCG on A^(k)
 * preconditioned by M^(k) (Section 4).  The loop continues to level 0
 * (A^(0) = A, M^(0) = I) so that the result meets a residual target.
 *
 * Conventions for every entry point:
 *   - Return value: MMD_OK (0) or a negative MMD_E* code; no exception or
 *     C++ type crosses the boundary.  mmd_strerror() names a code and
 *     mmd_last_error() gives a message for the calling thread's last failure.
 *   - Sparse input: full symmetric CSR storage (both triangles), int32 row
 *     pointers and column indices sorted ascending within each row, FP64
 *     values, diagonal present.  Pointers are host memory unless the struct's
 *     on_device flag is 1 (device memory of the current CUDA device).
 *     Inputs are borrowed for the duration of the call only.
 *   - Dense outputs are caller-allocated, column-major.  *_on_device flags say
 *     whether an output pointer is device memory.
 *   - Streams: work is enqueued on the cudaStream_t passed as void*
 *     (NULL = legacy default stream); every entry point synchronises that
 *     stream before it returns.
 *   - Handles are not thread-safe: one call at a time per handle.
 */
#ifndef MMDEIG_H
#define MMDEIG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MMD_OK 0
#define MMD_EINVAL (-1)   /* bad argument or malformed CSR */
#define MMD_ENOTSPD (-2)  /* a Cholesky/energy found a non-SPD matrix */
#define MMD_ENOCONV (-3)  /* an iteration cap was hit; partial results returned */
#define MMD_ETIMEOUT (-4) /* a device-side wait exceeded its time limit */
#define MMD_ECUDA (-5)    /* a CUDA runtime call failed */
#define MMD_ENOMEM (-6)   /* host or device allocation failed */

/* methods of eig_leftmost */
#define MMD_HIERARCHICAL 0 /* Algorithm 6 on the decomposition (the paper's method) */
#define MMD_IRLM_CG 1      /* Section 8's baseline: implicitly restarted Lanczos on A^{-1}, each
                              application by plain CG (or the polynomial PCG of poly_op when
                              that is set), no decomposition (the extension of
                              Algorithm 4 at level 0 from an empty basis with searching step
                              d = N, i.e. N wanted and N shifts per restart) */

/* precision modes of eig_leftmost */
#define MMD_FP64 0      /* every step in FP64 */
#define MMD_MIXED 1     /* coarse levels k >= 1: FP32 PCG inside FP64 iterative
                           refinement; level-0 CG on A in double-float arithmetic
                           (FP32 pairs, ~48 bits) with its FP64 residual checked
                           before a column is accepted (FP64 CG finishes a column
                           it cannot); all dense work in FP64 */
#define MMD_MIXED_ALL 2 /* as MMD_MIXED, and level-0 CG with FP32 recurrences and
                           FP64 reliable updates (for kappa(A) well below 1/u_32) */

typedef struct mmd_handle mmd_handle;

typedef struct {
  int64_t n;             /* rows = columns */
  int64_t nnz;           /* stored entries (both triangles) */
  const int32_t* rowptr; /* n + 1 */
  const int32_t* col;    /* nnz, ascending per row */
  const double* val;     /* nnz */
  int on_device;         /* 1: the three arrays are device pointers */
} mmd_csr;

/* Decomposition build options (the patch construction is this library's
 * reading of Section 2.2: integer-only aggregation of the matrix pattern,
 * interior-energy phi, localized psi on whole neighbouring patches). */
typedef struct {
  int s_max;      /* pass-1 patch size cap; joins allowed up to 2*s_max (default 8) */
  int omega_max;  /* row cap of a psi support neighbourhood (default 256) */
  int loc_radius; /* 0: support = own patch, r >= 1: plus r rings of neighbouring patches
                     (default 1; r > 1 at level 1 only, deeper levels use one ring) */
  int n_coarse;   /* stop when N^(k) <= n_coarse (default 300) */
  int k_max;      /* maximum number of levels (default 8) */
  int device;     /* 1: upload the levels to the current CUDA device (default);
                     0: host-only handle (inspection with mmd_level_info only) */
  int threads;    /* host threads for the build, 0 = all cores */
  double peel;    /* > 0: split weakly attached rows off a patch while its 1/lambda_2
                     exceeds peel x the median over patches (bounds eps(P)); 0 = off */
  int gpu_psi;    /* 1: with device = 1, the local psi solves of every level (Section 2.2's
                     energy-minimising basis on each support, one dense KKT system per patch,
                     independent across patches) run on the GPU, one block per patch; the
                     integer indexing is the host's either way (default 1) */
} mmd_build_opts;

/* Solver options (Section 6 parameter rules). */
typedef struct {
  double alpha;        /* refinement threshold mu_re^(k) = alpha eps_{k+1} (default 3) */
  double beta;         /* extension threshold mu_ex^(k) = beta eps_k (default 1) */
  int d;               /* searching step, 0 = min(N^(k)/10, N/10) clamped to >= 1 */
  int c_r;             /* restart factor: p = c_r * d shifts (default 1) */
  int precision;       /* MMD_FP64, MMD_MIXED or MMD_MIXED_ALL */
  int max_cg_iter;     /* cap per CG/PCG call (default 20000) */
  int max_restarts;    /* cap per convergence loop (default 400) */
  int max_refine_iter; /* cap of Algorithm 5 iterations (default 100) */
  double timeout_s;    /* per device-side wait (default 2 s) */
  uint64_t seed;       /* SplitMix64 seed of the random vectors drawn */
  void* stream;        /* cudaStream_t */
  int profile;         /* 1: time every launch of the PCG kernel with events */
  int method;          /* MMD_HIERARCHICAL (default) or MMD_IRLM_CG */
  int stop_level;      /* MMD_HIERARCHICAL: the last level Algorithm 6 computes (default 0: the
                          level-0 completion, residual target tol).  s >= 1 ends at level s with
                          its own accuracy eps_s (Lemma 3.3) and returns V = Psi^(1)...Psi^(s) V^(s):
                          s = 1 is Algorithm 6's own output, s = K the dense solve of the coarsest
                          pencil (Section 7.2); the last level extends to N pairs without the
                          extension threshold.  Must be <= K. */
  int mg_refine;       /* level-0 refinement solves (Algorithm 5, warm-started PCG on A) use the
                          decomposition as a preconditioner (Section 2.3's A^{-1} representation
                          applied as an FP32 V-cycle over the levels, Chebyshev smoothing of this
                          degree; the outer PCG stays FP64 with the same stopping test).  0 = plain
                          CG.  Default 2. */
  int mg_op;           /* the same preconditioner, with this Chebyshev degree, for the level-0 solves
                          of Operator OP inside the Lanczos extension (Algorithm 4 at level 0, where
                          M^(0) = I leaves plain CG on A); OP's result, A^{-1}x to the same relative
                          residual, is unchanged.  0 = plain CG.  MMD_IRLM_CG always uses plain CG. */
  int poly_op;         /* level-0 Operator OP solves (Lanczos extension, and MMD_IRLM_CG's solves) by
                          FP64 flexible PCG preconditioned by p(D^{-1}A) D^{-1}: this many steps of the
                          Chebyshev iteration for A z = r on the interval [hi / poly_ratio, hi] of
                          D^{-1}A (hi its Gershgorin bound), in FP32.  Same result (A^{-1}x to the same
                          relative residual); trades grid-wide reductions and FP64 SpMVs for FP32 SpMVs.
                          0 = off (plain CG, the default); takes precedence over mg_op.  <= 32. */
  int poly_refine;     /* the same for the level-0 refinement solves; takes precedence over
                          mg_refine.  0 = off (default). */
  double poly_ratio;   /* hi / lo of the polynomial's interval (default 1000) */
} mmd_eig_opts;

/* Counters and timings of one eig_leftmost call (Section 7 reports the same
 * kinds of counters: PCG/CG calls and iterations, refinement iterations). */
typedef struct {
  int64_t op_calls, pcg_iters, inner_iters;      /* Operator OP (Alg 3 line 7) */
  int64_t b_calls, b_iters;                      /* CG on B^(k) (Alg 5) */
  int64_t refine_pcg_calls, refine_pcg_iters;    /* warm-started PCG in Alg 5 */
  int64_t restarts, lanczos_steps, refine_iters; /* Alg 2, Alg 3, Alg 5 */
  int64_t not_converged;                         /* capped loops (sum of the three below) */
  int64_t nc_solve, nc_restart, nc_refine;       /* capped CG/PCG solves, restart loops, refinements */
  int64_t kernel_launches;                       /* CUDA kernels launched */
  int n_levels;                                  /* K + 1 */
  int n_converged;                               /* pairs meeting the residual target */
  double norm_A;                                 /* ||A||_inf, upper bound of ||A||_2 */
  double max_rel_residual;                       /* max ||Av - lv||_2 / ||A||_inf */
  double mu1;                                    /* largest mu found on the coarsest level */
  double t_total_ms;
  /* profile == 1: the sparse-solver kernel's launches */
  int64_t pcg_launches;
  double pcg_ms;        /* sum of event-timed durations */
  double pcg_bytes;     /* algorithmic bytes moved by those launches */
  double pcg_flops;     /* algorithmic floating-point operations of those launches */
  int64_t fp64_finishes; /* MMD_MIXED_ALL: level-0 CG columns FP32 left unconverged, finished in FP64 */
  double t_level_ms[16]; /* wall time per level k (coarsest solve; refinement + extension) */
  /* profile == 1: the subset of those launches that are level-0 Operator OP solves (CG on A,
     one column: the extension's Lanczos steps) */
  int64_t op0_launches;
  double op0_ms, op0_bytes, op0_flops;
  int64_t op0_iters;
  /* per level k: the most iterations one PCG call on A^(k) took (the extension's Operator OP
     and the refinement's warm-started solves; Section 7's #^(A^(k))) */
  int64_t max_pcg_iters[16];
  /* launches of the wide multi-column solve (MMD_MIXED, level-0 blocks of >= 8 columns) replayed
     from the CUDA graph captured at its first call with the same buffers */
  int64_t graph_replays;
} mmd_eig_stats;

/* Read-only view of level k (1 <= k <= K) of a handle; host pointers owned by
 * the handle, valid until mmd_free.  Arrays follow the natural (build) order:
 * patches in creation order, rows ascending within a patch. */
typedef struct {
  int64_t n_fine;            /* N^(k-1) */
  int64_t n;                 /* N^(k) = number of patches */
  const int32_t* patch_of;   /* n_fine */
  const int32_t* patch_ptr;  /* n + 1 */
  const int32_t* patch_rows; /* n_fine */
  const double* phi;         /* n_fine, aligned with patch_rows */
  const int32_t* omega_ptr;  /* n + 1: support of psi_j */
  const int32_t* omega_rows; /* omega_ptr[n] */
  int64_t psi_nnz;           /* Psi^(k): N^(k-1) x N^(k), CSR */
  const int32_t* psi_rowptr;
  const int32_t* psi_col;
  const double* psi_val;
  int64_t a_nnz;             /* A^(k), CSR */
  const int32_t* a_rowptr;
  const int32_t* a_col;
  const double* a_val;
  int64_t m_nnz;             /* M^(k), CSR */
  const int32_t* m_rowptr;
  const int32_t* m_col;
  const double* m_val;
  double eps;                /* error factor eps(P^(k)), Section 2.2 */
  double delta;              /* condition factor delta(P^(k)), Theorem 2.2 */
  int used_closed;           /* patches whose interior energy was not PSD */
} mmd_level_view;

void mmd_default_build_opts(mmd_build_opts* o);
void mmd_default_eig_opts(mmd_eig_opts* o);

/* Build the decomposition of A (Section 2.3).  A is copied; *out owns every
 * level (host arrays, and device arrays when opts->device = 1).
 * Errors: MMD_EINVAL (n < 1, unsorted/duplicate/out-of-range columns, missing
 * diagonal, asymmetric pattern or values), MMD_ENOTSPD (a local energy or
 * neighbourhood matrix is not positive definite), MMD_ENOMEM, MMD_ECUDA. */
int mmd_build(const mmd_csr* A, const mmd_build_opts* opts, mmd_handle** out);

/* Number of levels K (the handle holds levels 0..K). */
int mmd_num_levels(const mmd_handle* h);

/* Size N^(k) of level k (0 <= k <= K), or a negative code. */
int64_t mmd_level_size(const mmd_handle* h, int k);

/* Fill *out with read-only views of level k, 1 <= k <= K. */
int mmd_level_info(const mmd_handle* h, int k, mmd_level_view* out);

/* N leftmost eigenpairs of A (Algorithm 6 with the level-0 completion).
 * tol: relative residual target ||A v - lambda v||_2 <= tol ||A||.
 * lambda: N values ascending; V: n x N column-major, 2-norm orthonormal
 * columns, sign so that the largest-|.| entry is positive.  lambda and V are
 * host or device memory per outputs_on_device.  stats may be NULL.
 * Requires a device handle.  MMD_ENOCONV returns the best pairs found. */
int eig_leftmost(mmd_handle* h, int N, double tol, const mmd_eig_opts* opts,
                 double* lambda, double* V, int outputs_on_device,
                 mmd_eig_stats* stats);

/* eig_leftmost on `count` independent problems at once (the data-parallel
 * use of Algorithm 6: one decomposition per graph).  hs[i], N[i], lambda[i],
 * V[i] and stats[i] (stats may be NULL) are those of problem i; tol and opts
 * are shared (opts->stream is ignored).  The problems run concurrently on
 * `streams` non-blocking CUDA streams (<= 0: 8), one host thread per stream;
 * the largest problems (n N) start first and each stream takes the next
 * problem when it is free.  Each stream's cooperative solver launches use at
 * most (SM count / streams) blocks, so the concurrent grids are co-resident.
 * The handles must be distinct.  Returns MMD_OK, or the first failing
 * problem's code (all problems are still attempted; mmd_last_error names the
 * problem). */
int eig_leftmost_batched(mmd_handle* const* hs, int count, const int* N, double tol, const mmd_eig_opts* opts,
                         double* const* lambda, double* const* V, int outputs_on_device,
                         mmd_eig_stats* stats, int streams);

/* Gradient of a loss L(lambda, V) of the last eig_leftmost result of h with
 * respect to the stored values of the input CSR (not in the paper; the
 * adjoint of the solver's output).  With (lambda_i, v_i), i < N, the pairs
 * returned by that call, gl = dL/dlambda (N) and Gv = dL/dV (n x N,
 * column-major, NULL when L depends on lambda only):
 *   dL/dval_e = sum_i [gl_i v_i(r_e) + y_i(r_e)] v_i(c_e),
 *   y_i = -(A - lambda_i I)^+ g_i  (first-order eigenvector perturbation),
 * where y_i = in-block terms sum_{j != i} v_j (v_j^T g_i)/(lambda_i - lambda_j)
 * plus the solution z of (A - lambda_i I) z = -(I - V V^T) g_i on the
 * complement of the block (conjugate gradients; needs lambda_i < lambda_{N+1}).
 * e runs over the stored entries in the input's CSR order; a symmetric pair
 * (r, c), (c, r) receives its two derivatives separately.  Assumes simple
 * eigenvalues for the pairs with nonzero Gv columns.  Inputs and the output
 * (nnz doubles) are device memory when the flags are 1.  Errors: MMD_EINVAL
 * (no previous result), MMD_ENOTSPD (lambda_i not below the complement). */
int eig_grad(mmd_handle* h, const double* dL_dlambda, const double* dL_dV, int inputs_on_device, double* dL_dvals,
             int output_on_device, const mmd_eig_opts* opts);

/* Level operators on device vectors of level k, in the natural (build) order
 * of that level, for tests and kernel benchmarks.
 * mmd_level_spmv: y = A^(k) x (which = 0) or M^(k) x (which = 1, k >= 1).
 * mmd_level_spmv_timed: the same product, computed reps times back to back
 *   on the level's device-order copy of x; *ms = mean time of one SpMV
 *   kernel between two events on the stream (the permutations of x and y
 *   stay outside the timed region).
 * mmd_level_op: y = OP(x) = pcg(A^(k), M^(k) x, M^(k), 0, tol) (the Operator
 *   OP box after Algorithm 3); k = 0 uses M = I (plain CG).  iters may be NULL.
 * mmd_level_op_block: Y = OP(X) for m columns (n_k x m, column-major), the
 *   warm-start-free form of the refinement's multi-right-hand-side PCG
 *   (Algorithm 5), 4 columns per solver launch; precision as in
 *   mmd_eig_opts; iters (m entries) may be NULL.
 * mmd_level_bsolve: x = U g where g = CG(B^(k), U^T M^(k-1) q, tol) and
 *   B^(k) = U^(k)^T A^(k-1) U^(k) (Algorithm 5, first loop); q and x are
 *   level-(k-1) vectors, 1 <= k <= K. */
int mmd_level_spmv(mmd_handle* h, int k, int which, const double* x, double* y, void* stream);
int mmd_level_spmv_timed(mmd_handle* h, int k, int which, const double* x, double* y, int reps, float* ms,
                         void* stream);
int mmd_level_op(mmd_handle* h, int k, const double* x, double* y, double tol, int max_iter,
                 int64_t* iters, void* stream);
int mmd_level_op_block(mmd_handle* h, int k, int m, const double* X, double* Y, double tol, int max_iter,
                       int64_t* iters, int precision, void* stream);
int mmd_level_bsolve(mmd_handle* h, int k, const double* q, double* x, double tol, int max_iter,
                     int64_t* iters, void* stream);
/* mmd_level_vcycle: Z = V(R) for m columns of level 0 (n x m, column-major,
 *   device memory, natural order): one application of the V-cycle
 *   preconditioner of mg_refine (Section 2.3's representation A^{-1} =
 *   U B^{-1} U^T + Psi (Psi^T A Psi)^{-1} Psi^T applied level by level:
 *   Chebyshev smoothing of degree deg (>= 1) with D^{-1} A^(k) on
 *   [hi / 30, hi], hi the Gershgorin bound, restriction Psi^T, recursion,
 *   prolongation Psi, smoothing again; the coarsest level by its dense
 *   inverse), FP32 arithmetic, FP64 in and out.  Needs K >= 1 and a coarsest
 *   level of at most 2048 rows (else MMD_EINVAL). */
int mmd_level_vcycle(mmd_handle* h, int m, const double* R, double* Z, int deg, void* stream);
/* mmd_level_poly: Z = p(D^{-1} A) D^{-1} R for m columns of level 0 (n x m,
 *   column-major, device memory, natural order): one application of the
 *   polynomial preconditioner of poly_op / poly_refine, i.e. deg (1..32)
 *   steps of the Chebyshev iteration for A Z = R from Z = 0 on the interval
 *   [hi / ratio, hi] of D^{-1} A (D = diag A, hi its Gershgorin bound;
 *   ratio in (1, 1e12]); FP32 arithmetic, FP64 in and out.  The paper has
 *   no counterpart: level 0 is plain CG in Section 4 (M^(0) = I), and this
 *   operator only changes how A^{-1} x is reached, not its value. */
int mmd_level_poly(mmd_handle* h, int m, const double* R, double* Z, int deg, double ratio, void* stream);

/* The SpMV autotuner: when a level matrix is uploaded the library times each
 * single-column SELL SpMV kernel variant on it (entries in flight per lane
 * 4 / 8 / 16, blocks of 128 / 256 / 512 threads, register bounds; five
 * launches each after a warm-up) and uses the fastest for that matrix.
 * Returns the chosen variant of A^(k) (which = 0) or M^(k) (which = 1, k >= 1)
 * and writes every variant's mean time in ms to ms_per_variant (MMD_SPMV_VARIANTS
 * entries) unless it is NULL; MMD_EINVAL on bad arguments. */
#define MMD_SPMV_VARIANTS 6
int mmd_spmv_tuning(const mmd_handle* h, int k, int which, float* ms_per_variant);

/* The solver autotuner: at mmd_build, for every level k < K that runs CG /
 * PCG solves and both tile widths (mt = 1 or 4 columns), the library times
 * 20 iterations of CG on A^(k) at each of MMD_TUNE_GRIDS candidate grids
 * (2 ... 152 blocks of 1024 threads, those that are resident and leave at
 * least 64 rows per block) and runs that level's solves on the fastest grid
 * (capped by the SMs a batched call or a concurrent tile lane may use).
 * Returns the chosen grid, writes the candidates to grids and their measured
 * microseconds per iteration to us_per_iter (0 = not tried) unless NULL;
 * MMD_EINVAL for a host-only handle, k outside [0, K) or mt not 1 / 4.  The
 * paper has no counterpart (its solves run on one CPU core). */
#define MMD_TUNE_GRIDS 8
int mmd_solver_tuning(const mmd_handle* h, int k, int mt, int* grids, float* us_per_iter);

void mmd_free(mmd_handle* h);
const char* mmd_strerror(int code);
const char* mmd_last_error(void);

/* ---- a solve that allocates nothing ----
 * The paper has no counterpart of this entry point; it exists for callers
 * that must not allocate device memory during a call: services that reserve
 * all GPU memory at start-up and treat a later cudaMalloc as a failure, loops
 * with latency budgets that cannot absorb the synchronisation an allocation
 * may cause, or frameworks that give the library only inputs and outputs.
 *
 * x = A^{-1} b by plain conjugate gradients (x0 = 0, stop at
 * ||b - A x||_2 <= tol ||b||_2 or max_iter), the same iteration the library
 * applies as Operator OP on level 0.  A is a device CSR (A->on_device = 1,
 * full symmetric storage, SPD); b and x are device vectors of length A->n.
 * All working memory (three vectors, reduction partials, barrier counter)
 * is a fixed array inside the library of about 8 MB per GPU, held from the
 * first load until the process exits, so n is limited to MMD_NOALLOC_MAX_N;
 * larger n returns MMD_EINVAL with a message.  The call makes no cudaMalloc
 * or cudaFree and calls no allocating library routine.
 * The first call on a device (with that device current) looks up the array's
 * device address once (first calls from several host threads are serialised);
 * make that first call before any stream capture.
 * Every call reuses the same array and keeps nothing from the last one:
 * before its kernel it clears, on its stream, what must start at zero (the
 * barrier counter and the status word); calls that can run concurrently on
 * the GPU (unordered streams) race on the array, so order them.  The call is
 * synchronous: it waits on its stream for the iteration count and status
 * before it returns.  iters may be NULL.  Returns MMD_OK, MMD_EINVAL,
 * MMD_ENOCONV (max_iter reached, x holds the last iterate), MMD_ENOTSPD,
 * MMD_ETIMEOUT or MMD_ECUDA. */
#define MMD_NOALLOC_MAX_N 262144
int mmd_cg_solve_noalloc(const mmd_csr* A, const double* b, double* x, double tol, int max_iter, int64_t* iters,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif
