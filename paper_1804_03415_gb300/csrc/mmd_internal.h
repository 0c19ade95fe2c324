// Internal structures of the mmdeig library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mmdeig.h"

namespace mmd {

// Host CSR matrix (int32 indices, sorted columns).
struct HCSR {
  int64_t nrows = 0, ncols = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
  int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// One level k >= 1 of the decomposition in natural (build) order.
struct HLevel {
  int64_t n_fine = 0, n = 0;
  std::vector<int32_t> patch_of, patch_ptr, patch_rows, omega_ptr, omega_rows;
  std::vector<double> phi, uhat;
  HCSR psi;  // n_fine x n
  HCSR A, M;
  double eps = 0, delta = 0;
  int used_closed = 0;
};

// Device CSR (device order) plus its SELL-32 copy (slices of 32 rows, rows
// sorted by length inside windows of 256, entries column-major in a slice).
struct DCSR {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  float* val2 = nullptr;     // 2 x nnz: each CSR value as the FP32 pair (hi, lo), value = hi + lo
  double mean_row = 0;
  int max_row = 0;
  int64_t nslices = 0, sell_nnz = 0;
  int32_t* s_ptr = nullptr;   // nslices + 1, offsets of the slices
  int32_t* s_len = nullptr;   // nslices, width of each slice
  int32_t* s_row = nullptr;   // 32 * nslices, row of each lane (-1 = padding)
  int32_t* s_col = nullptr;   // sell_nnz
  double* s_val = nullptr;    // sell_nnz
  float* s_val32 = nullptr;   // sell_nnz
  float* s_val2 = nullptr;    // 2 x sell_nnz: each value as the pair (hi, lo) of FP32 numbers, value = hi + lo
  int spmv_variant = -1;      // single-column SpMV kernel chosen by the autotuner at upload
  std::vector<float> spmv_ms; // its timing of every variant (ms)
};

// Device level data.  Level k's vectors are stored in "device order": the
// rows of level k sorted by the patches of level k + 1 (patch by patch, so
// each patch of level k + 1 is a contiguous segment); the coarsest level keeps
// its natural order.
struct DLevel {
  int64_t n = 0;
  DCSR A;          // A^(k)
  DCSR M;          // M^(k), k >= 1
  DCSR psi;        // Psi^(k): level k-1 (rows) x level k (cols), k >= 1
  // patches of level k+1 over this level's rows (k < K): contiguous segments
  int64_t nseg = 0;
  int32_t* seg_ptr = nullptr;  // nseg + 1
  double* phi_next = nullptr;  // phi^(k+1) per row of this level (device order)
  std::vector<int32_t> perm;   // device position -> natural index (host copy)
  int32_t* d_perm = nullptr;   // same on device
  int32_t* d_iperm = nullptr;  // natural index -> device position
  double eps = 0, delta = 0;   // of P^(k) (k >= 1)
  // V-cycle preconditioner data (present when the handle's mg_ok is set)
  DCSR psiT;                   // (Psi^(k))^T: level k (rows) x level k-1 (cols), k >= 1
  float* dinv32 = nullptr;     // 1 / diag A^(k), k < K
  double gersh = 0;            // max_i sum_j |a_ij| / a_ii of A^(k), k < K
  float* kinv32 = nullptr;     // k = K: (A^(K))^{-1}, dense N^(K) x N^(K)
  // grid of the persistent solver for tiles of 1 and 4 columns, chosen by the
  // autotuner at build (0: not tuned, the size heuristic applies), with every
  // candidate's measured time per CG iteration (us; 0: candidate not tried)
  int grid[2] = {0, 0};
  float grid_us[2][8] = {};
};

struct Workspace;

}  // namespace mmd

struct mmd_handle {
  mmd::HCSR A0;                      // input, natural order
  std::vector<mmd::HLevel> levels;   // k = 1..K at index k-1
  mmd_build_opts bopts;
  bool on_device = false;
  int device = -1;
  std::vector<mmd::DLevel> dl;       // k = 0..K
  mmd::Workspace* ws = nullptr;
  double normA_inf = 0;
  // last eig_leftmost result (for eig_grad): eigenvalues ascending (host),
  // eigenvectors in natural order in the workspace buffer "last_V"
  std::vector<double> last_lam;
  int last_N = 0;
  int32_t* d_in_rowptr = nullptr;  // input CSR pattern (natural order), uploaded by eig_grad
  int32_t* d_in_col = nullptr;
  bool mg_ok = false;  // V-cycle data uploaded (K >= 1 and a dense-invertible coarsest level)
};

namespace mmd {

void set_error(const std::string& msg);
int build_host(const mmd_csr* A, const mmd_build_opts* o, mmd_handle* h);
int upload_levels(mmd_handle* h);
void free_device(mmd_handle* h);

}  // namespace mmd
