// C ABI of the library: handles, device upload, level operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "driver.h"
#include "kernels.h"
#include "mmd_internal.h"

namespace mmd {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

template <typename T>
static int dalloc(T** p, size_t n) {
  if (n == 0) n = 1;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
    return MMD_ENOMEM;
  }
  return MMD_OK;
}

template <typename T>
static int dput(T** p, const std::vector<T>& v) {
  int rc = dalloc(p, v.size());
  if (rc) return rc;
  if (!v.empty() && cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("cudaMemcpy to device failed");
    return MMD_ECUDA;
  }
  return MMD_OK;
}

// Permute a square CSR symmetrically: new row i' = old perm[i'], columns by iperm.
static HCSR permute_sym(const HCSR& A, const std::vector<int32_t>& perm, const std::vector<int32_t>& iperm) {
  HCSR B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rowptr.assign(A.nrows + 1, 0);
  for (int64_t i = 0; i < A.nrows; ++i) B.rowptr[i + 1] = B.rowptr[i] + (A.rowptr[perm[i] + 1] - A.rowptr[perm[i]]);
  B.col.resize(A.col.size());
  B.val.resize(A.val.size());
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < A.nrows; ++i) {
    const int32_t r = perm[i];
    row.clear();
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) row.push_back({iperm[A.col[k]], A.val[k]});
    std::sort(row.begin(), row.end());
    for (size_t t = 0; t < row.size(); ++t) {
      B.col[B.rowptr[i] + t] = row[t].first;
      B.val[B.rowptr[i] + t] = row[t].second;
    }
  }
  return B;
}

// Rows permuted by prow (new i' = old prow[i']), columns renumbered by icol.
static HCSR permute_rect(const HCSR& A, const std::vector<int32_t>& prow, const std::vector<int32_t>& icol) {
  HCSR B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rowptr.assign(A.nrows + 1, 0);
  for (int64_t i = 0; i < A.nrows; ++i) B.rowptr[i + 1] = B.rowptr[i] + (A.rowptr[prow[i] + 1] - A.rowptr[prow[i]]);
  B.col.resize(A.col.size());
  B.val.resize(A.val.size());
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < A.nrows; ++i) {
    const int32_t r = prow[i];
    row.clear();
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) row.push_back({icol[A.col[k]], A.val[k]});
    std::sort(row.begin(), row.end());
    for (size_t t = 0; t < row.size(); ++t) {
      B.col[B.rowptr[i] + t] = row[t].first;
      B.val[B.rowptr[i] + t] = row[t].second;
    }
  }
  return B;
}

// Pick the single-column SpMV kernel of this matrix by timing every variant
// on it (the autotuner; a few launches per variant on scratch vectors).
static int autotune_spmv(DCSR& D) {
  if (D.nrows < 1 || D.ncols < 1) return MMD_OK;
  double *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, sizeof(double) * D.ncols) != cudaSuccess ||
      cudaMalloc(&y, sizeof(double) * D.nrows) != cudaSuccess) {
    cudaFree(x);
    cudaGetLastError();
    set_error("cudaMalloc of the SpMV autotuner's vectors failed");
    return MMD_ENOMEM;
  }
  cudaMemset(x, 0, sizeof(double) * D.ncols);
  Sell s;
  s.nrows = D.nrows;
  s.nslices = D.nslices;
  s.ptr = D.s_ptr;
  s.len = D.s_len;
  s.row = D.s_row;
  s.col = D.s_col;
  s.val = D.s_val;
  s.val32 = D.s_val32;
  D.spmv_ms.assign(k_spmv_variants(), 0.f);
  D.spmv_variant = k_spmv_autotune(s, x, y, nullptr, D.spmv_ms.data());
  cudaFree(x);
  cudaFree(y);
  if (cudaDeviceSynchronize() != cudaSuccess || D.spmv_variant < 0) {
    set_error("the SpMV autotuner's launches failed");
    return MMD_ECUDA;
  }
  return MMD_OK;
}

static int upload_csr(const HCSR& A, DCSR& D) {
  D.nrows = A.nrows;
  D.ncols = A.ncols;
  D.nnz = A.nnz();
  int rc;
  if ((rc = dput(&D.rowptr, A.rowptr))) return rc;
  if ((rc = dput(&D.col, A.col))) return rc;
  if ((rc = dput(&D.val, A.val))) return rc;
  std::vector<float> v32(A.val.begin(), A.val.end());
  if ((rc = dput(&D.val32, v32))) return rc;
  std::vector<float> v2(2 * A.val.size());
  for (size_t i = 0; i < A.val.size(); ++i) {
    v2[2 * i] = v32[i];
    v2[2 * i + 1] = (float)(A.val[i] - (double)v32[i]);
  }
  if ((rc = dput(&D.val2, v2))) return rc;
  D.mean_row = A.nrows ? double(D.nnz) / double(A.nrows) : 0.0;
  int mx = 0;
  for (int64_t i = 0; i < A.nrows; ++i) mx = std::max(mx, A.rowptr[i + 1] - A.rowptr[i]);
  D.max_row = mx;
  // SELL-32: rows sorted by length (descending, stable) inside windows of 1024,
  // slices of 32 rows stored column-major, padded with zeros (column = row).
  const int64_t n = A.nrows, ns = (n + 31) / 32;
  std::vector<int32_t> order(n);
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  constexpr int64_t kSigma = 1024;  // torus kNN 200k: 1.2% padding (256: 4.2%, 32: 29%)
  for (int64_t w0 = 0; w0 < n; w0 += kSigma) {
    const int64_t w1 = std::min<int64_t>(n, w0 + kSigma);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) {
      return (A.rowptr[a + 1] - A.rowptr[a]) > (A.rowptr[b + 1] - A.rowptr[b]);
    });
  }
  std::vector<int32_t> sptr(ns + 1, 0), slen(ns, 0), srow(ns * 32, -1);
  for (int64_t s = 0; s < ns; ++s) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t t = s * 32 + l;
      if (t < n) {
        srow[t] = order[t];
        w = std::max(w, A.rowptr[order[t] + 1] - A.rowptr[order[t]]);
      }
    }
    slen[s] = w;
    if (int64_t(sptr[s]) + int64_t(w) * 32 >= (int64_t(1) << 31)) {
      set_error("SELL copy exceeds 2^31 entries");
      return MMD_EINVAL;
    }
    sptr[s + 1] = sptr[s] + w * 32;
  }
  const int64_t tot = sptr[ns];
  std::vector<int32_t> scol(tot);
  std::vector<double> sval(tot, 0.0);
  for (int64_t s = 0; s < ns; ++s)
    for (int l = 0; l < 32; ++l) {
      const int32_t r = srow[s * 32 + l];
      const int32_t k0 = r >= 0 ? A.rowptr[r] : 0, len = r >= 0 ? A.rowptr[r + 1] - k0 : 0;
      for (int k = 0; k < slen[s]; ++k) {
        const int64_t o = sptr[s] + int64_t(k) * 32 + l;
        if (k < len) {
          scol[o] = A.col[k0 + k];
          sval[o] = A.val[k0 + k];
        } else {
          scol[o] = r >= 0 ? std::min<int32_t>(r, (int32_t)A.ncols - 1) : 0;
          sval[o] = 0.0;
        }
      }
    }
  D.nslices = ns;
  D.sell_nnz = tot;
  if ((rc = dput(&D.s_ptr, sptr))) return rc;
  if ((rc = dput(&D.s_len, slen))) return rc;
  if ((rc = dput(&D.s_row, srow))) return rc;
  if ((rc = dput(&D.s_col, scol))) return rc;
  if ((rc = dput(&D.s_val, sval))) return rc;
  std::vector<float> sv32(sval.begin(), sval.end());
  if ((rc = dput(&D.s_val32, sv32))) return rc;
  std::vector<float> sv2(2 * tot);
  for (int64_t i = 0; i < tot; ++i) {
    const float hi = (float)sval[i];
    sv2[2 * i] = hi;
    sv2[2 * i + 1] = (float)(sval[i] - (double)hi);
  }
  if ((rc = dput(&D.s_val2, sv2))) return rc;
  return autotune_spmv(D);
}

// largest coarsest level whose dense inverse is formed for the V-cycle
constexpr int64_t kMgMaxCoarse = 2048;

static HCSR transpose(const HCSR& A) {
  HCSR T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.rowptr.assign(T.nrows + 1, 0);
  for (int32_t c : A.col) ++T.rowptr[c + 1];
  for (int64_t i = 0; i < T.nrows; ++i) T.rowptr[i + 1] += T.rowptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int32_t> fill(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int64_t r = 0; r < A.nrows; ++r)  // rows ascending: columns of T come out sorted
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      const int32_t o = fill[A.col[k]]++;
      T.col[o] = (int32_t)r;
      T.val[o] = A.val[k];
    }
  return T;
}

// max_i sum_j |a_ij| / a_ii: the Gershgorin bound of lambda_max(D^{-1} A)
static double gershgorin(const HCSR& A) {
  double g = 0;
  for (int64_t r = 0; r < A.nrows; ++r) {
    double s = 0, d = 0;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      s += std::fabs(A.val[k]);
      if (A.col[k] == r) d = A.val[k];
    }
    if (d > 0) g = std::max(g, s / d);
  }
  return g;
}

// Dense inverse of the SPD matrix A (n <= a few thousand) by Cholesky
// A = L L^T and n solves; false when a pivot is not positive.
static bool spd_inverse(const HCSR& A, std::vector<double>& inv) {
  const int64_t n = A.nrows;
  std::vector<double> L(size_t(n) * n, 0.0);  // row-major lower triangle
  for (int64_t r = 0; r < n; ++r)
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k)
      if (A.col[k] <= r) L[size_t(r) * n + A.col[k]] = A.val[k];
  for (int64_t j = 0; j < n; ++j) {
    double d = L[size_t(j) * n + j];
    for (int64_t k = 0; k < j; ++k) d -= L[size_t(j) * n + k] * L[size_t(j) * n + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    L[size_t(j) * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = L[size_t(i) * n + j];
      for (int64_t k = 0; k < j; ++k) t -= L[size_t(i) * n + k] * L[size_t(j) * n + k];
      L[size_t(i) * n + j] = t / d;
    }
  }
  inv.assign(size_t(n) * n, 0.0);
  std::vector<double> y(n);
  for (int64_t c = 0; c < n; ++c) {  // column c of A^{-1}: L y = e_c, L^T x = y
    for (int64_t i = 0; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) t -= L[size_t(i) * n + k] * y[k];
      y[i] = t / L[size_t(i) * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int64_t k = i + 1; k < n; ++k) t -= L[size_t(k) * n + i] * inv[size_t(c) * n + k];
      inv[size_t(c) * n + i] = t / L[size_t(i) * n + i];
    }
  }
  return true;
}

static void free_csr(DCSR& D) {
  cudaFree(D.rowptr);
  cudaFree(D.col);
  cudaFree(D.val);
  cudaFree(D.val32);
  cudaFree(D.val2);
  cudaFree(D.s_ptr);
  cudaFree(D.s_len);
  cudaFree(D.s_row);
  cudaFree(D.s_col);
  cudaFree(D.s_val);
  cudaFree(D.s_val32);
  cudaFree(D.s_val2);
  D = DCSR();
}

int upload_levels(mmd_handle* h) {
  const int K = (int)h->levels.size();
  h->dl.assign(K + 1, DLevel());
  // device order of level k: patches of level k+1 (natural patch ids), rows ascending inside
  std::vector<std::vector<int32_t>> perm(K + 1), iperm(K + 1);
  for (int k = 0; k <= K; ++k) {
    const int64_t n = (k == 0) ? h->A0.nrows : h->levels[k - 1].n;
    if (k < K)
      perm[k] = h->levels[k].patch_rows;
    else {
      perm[k].resize(n);
      for (int64_t i = 0; i < n; ++i) perm[k][i] = (int32_t)i;
    }
    iperm[k].resize(n);
    for (int64_t i = 0; i < n; ++i) iperm[k][perm[k][i]] = (int32_t)i;
  }
  int rc;
  for (int k = 0; k <= K; ++k) {
    DLevel& L = h->dl[k];
    const HCSR& A = (k == 0) ? h->A0 : h->levels[k - 1].A;
    L.n = A.nrows;
    if ((rc = upload_csr(permute_sym(A, perm[k], iperm[k]), L.A))) return rc;
    if (k >= 1) {
      const HLevel& H = h->levels[k - 1];
      if ((rc = upload_csr(permute_sym(H.M, perm[k], iperm[k]), L.M))) return rc;
      if ((rc = upload_csr(permute_rect(H.psi, perm[k - 1], iperm[k]), L.psi))) return rc;
      L.eps = H.eps;
      L.delta = H.delta;
    }
    if (k < K) {
      const HLevel& N = h->levels[k];
      L.nseg = N.n;
      if ((rc = dput(&L.seg_ptr, N.patch_ptr))) return rc;
      if ((rc = dput(&L.phi_next, N.phi))) return rc;
    }
    L.perm = perm[k];
    if ((rc = dput(&L.d_perm, perm[k]))) return rc;
    if ((rc = dput(&L.d_iperm, iperm[k]))) return rc;
  }
  // 1 / diag (FP32, device order) and the Gershgorin bound of D^{-1} A^(k):
  // level 0 always (the polynomial preconditioner of the level-0 solves),
  // the other smoothed levels with the V-cycle
  auto diag_data = [&](int k) -> int {
    DLevel& L = h->dl[k];
    if (L.dinv32) return MMD_OK;
    const HCSR& A = (k == 0) ? h->A0 : h->levels[k - 1].A;
    L.gersh = gershgorin(A);
    std::vector<float> dinv(A.nrows);
    for (int64_t i = 0; i < A.nrows; ++i) {
      const int32_t r = perm[k][i];
      double d = 0;
      for (int32_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e)
        if (A.col[e] == r) d = A.val[e];
      dinv[i] = (float)(1.0 / d);
    }
    return dput(&L.dinv32, dinv);
  };
  if ((rc = diag_data(0))) return rc;
  // V-cycle preconditioner of the level-0 refinement solves: Psi^T per level,
  // 1 / diag and the Gershgorin bound per smoothed level, the coarsest inverse
  h->mg_ok = false;
  const int64_t nK = h->dl[K].n;
  if (K >= 1 && nK <= kMgMaxCoarse) {
    std::vector<double> inv;
    const HCSR& AK = h->levels[K - 1].A;
    if (spd_inverse(AK, inv)) {
      for (int k = 0; k < K; ++k) {
        if ((rc = diag_data(k))) return rc;
        const HLevel& H = h->levels[k];
        if ((rc = upload_csr(transpose(permute_rect(H.psi, perm[k], iperm[k + 1])), h->dl[k + 1].psiT))) return rc;
      }
      std::vector<float> kinv(inv.begin(), inv.end());  // natural order = device order on level K
      if ((rc = dput(&h->dl[K].kinv32, kinv))) return rc;
      h->mg_ok = true;
    }
  }
  return MMD_OK;
}

void free_device(mmd_handle* h) {
  for (auto& L : h->dl) {
    free_csr(L.A);
    free_csr(L.M);
    free_csr(L.psi);
    free_csr(L.psiT);
    cudaFree(L.dinv32);
    cudaFree(L.kinv32);
    cudaFree(L.seg_ptr);
    cudaFree(L.phi_next);
    cudaFree(L.d_perm);
    cudaFree(L.d_iperm);
  }
  h->dl.clear();
  cudaFree(h->d_in_rowptr);
  cudaFree(h->d_in_col);
  h->d_in_rowptr = nullptr;
  h->d_in_col = nullptr;
  free_workspace(h);
}

}  // namespace mmd

using namespace mmd;

extern "C" {

void mmd_default_build_opts(mmd_build_opts* o) {
  if (!o) return;
  o->s_max = 8;
  o->omega_max = 256;
  o->loc_radius = 1;
  o->n_coarse = 300;
  o->k_max = 8;
  o->device = 1;
  o->threads = 0;
  o->peel = 0.0;
  o->gpu_psi = 1;
}

void mmd_default_eig_opts(mmd_eig_opts* o) {
  if (!o) return;
  o->alpha = 3.0;
  o->beta = 1.0;
  o->d = 0;
  o->c_r = 1;
  o->precision = MMD_FP64;
  o->max_cg_iter = 20000;
  o->max_restarts = 400;
  o->max_refine_iter = 100;
  o->timeout_s = 2.0;
  o->seed = 20180409ull;
  o->stream = nullptr;
  o->profile = 0;
  o->method = MMD_HIERARCHICAL;
  o->stop_level = 0;
  o->mg_refine = 2;
  o->mg_op = 0;
  o->poly_op = 0;
  o->poly_refine = 0;
  o->poly_ratio = 1000.0;
}

int mmd_build(const mmd_csr* A, const mmd_build_opts* opts, mmd_handle** out) {
  if (!out) {
    set_error("mmd_build: out is NULL");
    return MMD_EINVAL;
  }
  *out = nullptr;
  mmd_build_opts o;
  mmd_default_build_opts(&o);
  if (opts) o = *opts;
  if (o.s_max < 1 || o.omega_max < 1 || o.n_coarse < 1 || o.k_max < 0 || o.loc_radius < 0 || !(o.peel >= 0) ||
      (o.gpu_psi != 0 && o.gpu_psi != 1)) {
    set_error("mmd_build: invalid build options");
    return MMD_EINVAL;
  }
  if (!A) {
    set_error("mmd_build: A is NULL");
    return MMD_EINVAL;
  }
  mmd_handle* h = new (std::nothrow) mmd_handle();
  if (!h) return MMD_ENOMEM;
  h->bopts = o;
  mmd_csr hostA = *A;
  std::vector<int32_t> rp, ci;
  std::vector<double> va;
  if (A->on_device) {
    if (A->n < 1 || A->nnz < 1) {
      delete h;
      set_error("mmd_build: bad sizes");
      return MMD_EINVAL;
    }
    rp.resize(A->n + 1);
    ci.resize(A->nnz);
    va.resize(A->nnz);
    if (cudaMemcpy(rp.data(), A->rowptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ci.data(), A->col, ci.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(va.data(), A->val, va.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete h;
      set_error("mmd_build: copying the device CSR failed");
      return MMD_ECUDA;
    }
    hostA.rowptr = rp.data();
    hostA.col = ci.data();
    hostA.val = va.data();
    hostA.on_device = 0;
  }
  int rc;
  try {
    rc = build_host(&hostA, &o, h);
  } catch (const std::bad_alloc&) {
    rc = MMD_ENOMEM;
    set_error("mmd_build: host allocation failed");
  }
  if (rc == MMD_OK && o.device) {
    h->on_device = true;
    cudaGetDevice(&h->device);
    rc = upload_levels(h);
    if (rc == MMD_OK) rc = tune_solver(h);
  }
  if (rc != MMD_OK) {
    mmd_free(h);
    return rc;
  }
  *out = h;
  return MMD_OK;
}

int mmd_num_levels(const mmd_handle* h) { return h ? (int)h->levels.size() : MMD_EINVAL; }

int64_t mmd_level_size(const mmd_handle* h, int k) {
  if (!h || k < 0 || k > (int)h->levels.size()) return MMD_EINVAL;
  return k == 0 ? h->A0.nrows : h->levels[k - 1].n;
}

int mmd_level_info(const mmd_handle* h, int k, mmd_level_view* v) {
  if (!h || !v || k < 1 || k > (int)h->levels.size()) {
    set_error("mmd_level_info: level out of range");
    return MMD_EINVAL;
  }
  const HLevel& L = h->levels[k - 1];
  v->n_fine = L.n_fine;
  v->n = L.n;
  v->patch_of = L.patch_of.data();
  v->patch_ptr = L.patch_ptr.data();
  v->patch_rows = L.patch_rows.data();
  v->phi = L.phi.data();
  v->omega_ptr = L.omega_ptr.data();
  v->omega_rows = L.omega_rows.data();
  v->psi_nnz = L.psi.nnz();
  v->psi_rowptr = L.psi.rowptr.data();
  v->psi_col = L.psi.col.data();
  v->psi_val = L.psi.val.data();
  v->a_nnz = L.A.nnz();
  v->a_rowptr = L.A.rowptr.data();
  v->a_col = L.A.col.data();
  v->a_val = L.A.val.data();
  v->m_nnz = L.M.nnz();
  v->m_rowptr = L.M.rowptr.data();
  v->m_col = L.M.col.data();
  v->m_val = L.M.val.data();
  v->eps = L.eps;
  v->delta = L.delta;
  v->used_closed = L.used_closed;
  return MMD_OK;
}

void mmd_free(mmd_handle* h) {
  if (!h) return;
  if (h->on_device) free_device(h);
  delete h;
}

const char* mmd_strerror(int code) {
  switch (code) {
    case MMD_OK: return "ok";
    case MMD_EINVAL: return "invalid argument";
    case MMD_ENOTSPD: return "matrix not symmetric positive definite";
    case MMD_ENOCONV: return "iteration cap reached before convergence";
    case MMD_ETIMEOUT: return "device wait timed out";
    case MMD_ECUDA: return "CUDA error";
    case MMD_ENOMEM: return "out of memory";
    default: return "unknown error";
  }
}

const char* mmd_last_error(void) { return g_last_error.c_str(); }

int mmd_level_spmv(mmd_handle* h, int k, int which, const double* x, double* y, void* stream) {
  if (!h || !h->on_device || k < 0 || k > (int)h->levels.size() || (which == 1 && k == 0) || !x || !y) {
    set_error("mmd_level_spmv: bad arguments");
    return MMD_EINVAL;
  }
  return level_spmv(h, k, which, x, y, (cudaStream_t)stream);
}

int mmd_level_spmv_timed(mmd_handle* h, int k, int which, const double* x, double* y, int reps, float* ms,
                         void* stream) {
  if (!h || !h->on_device || k < 0 || k > (int)h->levels.size() || (which != 0 && which != 1) ||
      (which == 1 && k == 0) || !x || !y || reps < 1 || !ms) {
    set_error("mmd_level_spmv_timed: bad arguments");
    return MMD_EINVAL;
  }
  return level_spmv_timed(h, k, which, x, y, reps, ms, (cudaStream_t)stream);
}

int mmd_level_op(mmd_handle* h, int k, const double* x, double* y, double tol, int max_iter, int64_t* iters,
                 void* stream) {
  if (!h || !h->on_device || k < 0 || k > (int)h->levels.size() || !x || !y || !(tol > 0) || max_iter < 1) {
    set_error("mmd_level_op: bad arguments");
    return MMD_EINVAL;
  }
  return level_op(h, k, x, y, tol, max_iter, iters, (cudaStream_t)stream);
}

int mmd_level_op_block(mmd_handle* h, int k, int m, const double* X, double* Y, double tol, int max_iter,
                       int64_t* iters, int precision, void* stream) {
  if (!h || !h->on_device || k < 0 || k > (int)h->levels.size() || m < 1 || !X || !Y || !(tol > 0) ||
      max_iter < 1 || (precision != MMD_FP64 && precision != MMD_MIXED && precision != MMD_MIXED_ALL)) {
    set_error("mmd_level_op_block: bad arguments");
    return MMD_EINVAL;
  }
  return level_op_block(h, k, m, X, Y, tol, max_iter, iters, precision, (cudaStream_t)stream);
}

int mmd_spmv_tuning(const mmd_handle* h, int k, int which, float* ms_per_variant) {
  if (!h || !h->on_device || k < 0 || k > (int)h->levels.size() || (which != 0 && which != 1) ||
      (which == 1 && k == 0)) {
    set_error("mmd_spmv_tuning: bad arguments");
    return MMD_EINVAL;
  }
  const DCSR& D = which ? h->dl[k].M : h->dl[k].A;
  if (ms_per_variant)
    for (size_t v = 0; v < D.spmv_ms.size(); ++v) ms_per_variant[v] = D.spmv_ms[v];
  return D.spmv_variant;
}

int mmd_solver_tuning(const mmd_handle* h, int k, int mt, int* grids, float* us_per_iter) {
  if (!h || !h->on_device || k < 0 || k >= (int)h->levels.size() || (mt != 1 && mt != 4)) {
    set_error("mmd_solver_tuning: bad arguments (device handle, 0 <= k < K, mt 1 or 4)");
    return MMD_EINVAL;
  }
  const int w = mt == 1 ? 0 : 1;
  for (int i = 0; i < 8; ++i) {
    if (grids) grids[i] = kTuneGrids[i];
    if (us_per_iter) us_per_iter[i] = h->dl[k].grid_us[w][i];
  }
  return h->dl[k].grid[w];
}

int mmd_level_vcycle(mmd_handle* h, int m, const double* R, double* Z, int deg, void* stream) {
  if (!h || !h->on_device || m < 1 || !R || !Z || deg < 1 || deg > 8) {
    set_error("mmd_level_vcycle: bad arguments");
    return MMD_EINVAL;
  }
  if (!h->mg_ok) {
    set_error("mmd_level_vcycle: the handle has no V-cycle (no coarse level, or a coarsest level above 2048 rows)");
    return MMD_EINVAL;
  }
  return level_vcycle(h, m, R, Z, deg, (cudaStream_t)stream);
}

int mmd_level_poly(mmd_handle* h, int m, const double* R, double* Z, int deg, double ratio, void* stream) {
  if (!h || !h->on_device || m < 1 || !R || !Z || deg < 1 || deg > 32 || !(ratio > 1.0) || !std::isfinite(ratio) ||
      ratio > 1e12) {
    set_error("mmd_level_poly: bad arguments");
    return MMD_EINVAL;
  }
  return level_poly(h, m, R, Z, deg, ratio, (cudaStream_t)stream);
}

int mmd_level_bsolve(mmd_handle* h, int k, const double* q, double* x, double tol, int max_iter, int64_t* iters,
                     void* stream) {
  if (!h || !h->on_device || k < 1 || k > (int)h->levels.size() || !q || !x || !(tol > 0) || max_iter < 1) {
    set_error("mmd_level_bsolve: bad arguments");
    return MMD_EINVAL;
  }
  return level_bsolve(h, k, q, x, tol, max_iter, iters, (cudaStream_t)stream);
}

// Options of eig_leftmost, eig_leftmost_batched and eig_grad: defaults when
// opts is NULL, else a copy checked field by field (values the algorithms
// cannot use are refused before any work starts).
static bool validated_opts(const mmd_eig_opts* opts, const char* who, mmd_eig_opts* out) {
  mmd_default_eig_opts(out);
  if (opts) *out = *opts;
  const mmd_eig_opts& o = *out;
  std::string bad;
  if (!(o.alpha > 0) || !std::isfinite(o.alpha)) bad = "alpha must be finite and > 0";
  else if (!(o.beta > 0) || !std::isfinite(o.beta)) bad = "beta must be finite and > 0";
  else if (o.c_r < 1) bad = "c_r must be >= 1";
  else if (o.d < 0) bad = "d must be >= 0";
  else if (o.max_cg_iter < 1 || o.max_restarts < 1 || o.max_refine_iter < 1) bad = "iteration caps must be >= 1";
  else if (!(o.timeout_s > 0) || !std::isfinite(o.timeout_s)) bad = "timeout_s must be finite and > 0";
  else if (o.precision != MMD_FP64 && o.precision != MMD_MIXED && o.precision != MMD_MIXED_ALL)
    bad = "precision must be MMD_FP64, MMD_MIXED or MMD_MIXED_ALL";
  else if (o.method != MMD_HIERARCHICAL && o.method != MMD_IRLM_CG)
    bad = "method must be MMD_HIERARCHICAL or MMD_IRLM_CG";
  else if (o.stop_level < 0 || o.stop_level > 16) bad = "stop_level must be in [0, K]";
  else if (o.method == MMD_IRLM_CG && o.stop_level != 0) bad = "stop_level applies to MMD_HIERARCHICAL only";
  else if (o.mg_refine < 0 || o.mg_refine > 8) bad = "mg_refine must be in [0, 8]";
  else if (o.mg_op < 0 || o.mg_op > 8) bad = "mg_op must be in [0, 8]";
  else if (o.poly_op < 0 || o.poly_op > 32 || o.poly_refine < 0 || o.poly_refine > 32)
    bad = "poly_op and poly_refine must be in [0, 32]";
  else if (!(o.poly_ratio > 1.0) || !std::isfinite(o.poly_ratio) || o.poly_ratio > 1e12)
    bad = "poly_ratio must be finite, > 1 and <= 1e12";
  if (!bad.empty()) {
    set_error(std::string(who) + ": invalid options: " + bad);
    return false;
  }
  return true;
}

int eig_leftmost(mmd_handle* h, int N, double tol, const mmd_eig_opts* opts, double* lambda, double* V,
                 int outputs_on_device, mmd_eig_stats* stats) {
  if (!h || !h->on_device) {
    set_error("eig_leftmost: needs a device handle");
    return MMD_EINVAL;
  }
  if (N < 1 || N > h->A0.nrows || !(tol > 0) || !lambda || !V) {
    set_error("eig_leftmost: N must be in [1, n], tol > 0, outputs non-NULL");
    return MMD_EINVAL;
  }
  mmd_eig_opts o;
  if (!validated_opts(opts, "eig_leftmost", &o)) return MMD_EINVAL;
  return run_eig(h, N, tol, o, lambda, V, outputs_on_device, stats);
}

int eig_leftmost_batched(mmd_handle* const* hs, int count, const int* N, double tol, const mmd_eig_opts* opts,
                         double* const* lambda, double* const* V, int outputs_on_device, mmd_eig_stats* stats,
                         int streams) {
  if (!hs || count < 1 || !N || !lambda || !V || !(tol > 0)) {
    set_error("eig_leftmost_batched: bad arguments");
    return MMD_EINVAL;
  }
  for (int i = 0; i < count; ++i)
    if (!hs[i] || !hs[i]->on_device || N[i] < 1 || N[i] > hs[i]->A0.nrows || !lambda[i] || !V[i]) {
      set_error("eig_leftmost_batched: problem " + std::to_string(i) + " has a bad handle, N or output");
      return MMD_EINVAL;
    }
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (hs[i] == hs[j]) {
        set_error("eig_leftmost_batched: problems " + std::to_string(j) + " and " + std::to_string(i) +
                  " share one handle (handles must be distinct: a handle serves one call at a time)");
        return MMD_EINVAL;
      }
  mmd_eig_opts o;
  if (!validated_opts(opts, "eig_leftmost_batched", &o)) return MMD_EINVAL;
  const int ns = std::max(1, std::min(count, streams > 0 ? streams : 8));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the streams' cooperative grids (one block per SM each) share the SMs
  const int cap = std::max(1, nsm / ns);
  std::vector<cudaStream_t> st(ns, nullptr);
  for (int t = 0; t < ns; ++t)
    if (cudaStreamCreateWithFlags(&st[t], cudaStreamNonBlocking) != cudaSuccess) {
      for (int u = 0; u < t; ++u) cudaStreamDestroy(st[u]);
      set_error("eig_leftmost_batched: stream creation failed");
      return MMD_ECUDA;
    }
  std::vector<int> rcs(count, MMD_OK);
  std::vector<std::string> msgs(count);
  // largest problems first, each stream taking the next one when it is free
  // (longest-processing-time-first list scheduling)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (int64_t)hs[a]->A0.nrows * N[a] > (int64_t)hs[b]->A0.nrows * N[b];
  });
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  for (int t = 0; t < ns; ++t)
    th.emplace_back([&, t]() {
      cudaSetDevice(dev);
      set_coop_grid_cap(cap);
      mmd_eig_opts ot = o;
      ot.stream = st[t];
      for (int q = next++; q < count; q = next++) {
        const int i = order[q];
        rcs[i] = run_eig(hs[i], N[i], tol, ot, lambda[i], V[i], outputs_on_device, stats ? &stats[i] : nullptr);
        if (rcs[i] != MMD_OK) msgs[i] = mmd_last_error();
      }
    });
  for (auto& x : th) x.join();
  for (int t = 0; t < ns; ++t) cudaStreamDestroy(st[t]);
  for (int i = 0; i < count; ++i)
    if (rcs[i] != MMD_OK) {
      set_error("eig_leftmost_batched: problem " + std::to_string(i) + ": " + msgs[i]);
      return rcs[i];
    }
  return MMD_OK;
}

int eig_grad(mmd_handle* h, const double* dL_dlambda, const double* dL_dV, int inputs_on_device, double* dL_dvals,
             int output_on_device, const mmd_eig_opts* opts) {
  if (!h || !h->on_device || !dL_dlambda || !dL_dvals) {
    set_error("eig_grad: needs a device handle, dL_dlambda and dL_dvals");
    return MMD_EINVAL;
  }
  if (h->last_N < 1) {
    set_error("eig_grad: call eig_leftmost on this handle first");
    return MMD_EINVAL;
  }
  mmd_eig_opts o;
  if (!validated_opts(opts, "eig_grad", &o)) return MMD_EINVAL;
  return run_grad(h, dL_dlambda, dL_dV, inputs_on_device, dL_dvals, output_on_device, o);
}

}  // extern "C"
