// Hierarchical Eigenpair Computation (Algorithm 6) on the device, with the
// Eigenpair Refinement (Algorithm 5), the Eigenpair Extension (Algorithm 4),
// the general M-Lanczos iteration (Algorithm 3), the implicit restart
// (Algorithm 2) and Operator OP.  Every vector and matrix operation runs in
// the library's kernels; the host keeps the control flow of the algorithms
// and reads back a few scalars per step (Ritz values, residual estimates,
// the subspace-change test).
//
// The readings of points the paper leaves open are those of the oracle:
//   * the loop of Algorithm 6 continues to level 0 (A^(0) = A, M^(0) = I);
//   * absolute thresholds in mu units; relative ones use eps_k / mu_1;
//     level 0 tests are relative to the residual target;
//   * Lanczos breakdown ||f||_M < 1e-10 ||w||_M draws a SplitMix64 vector;
//   * CGS2 re-orthogonalisation against [V_ini, V] in the M inner product;
//   * exact shifts after the p-step extension, p = max(c_r d, k) (k = current
//     dimension: the factorisation doubles before the shifts);
//   * refinement window: mu_mh >= max(mu_re, mu_ml alpha / (1 + beta));
//   * column-scaled CholQR2 for the M-QR, S symmetrised, stop test
//     ||Q_mh - Q'_mh (Q'_mh^T M Q_mh)||_F < eps / sqrt(1 + eps_h delta_h).
// Differences from the paper's own CPU design (same mathematics):
//   * CG on B = U^T A U runs in the coordinates x = U g, where U U^T is the
//     per-patch projector I - phi phi^T (no Householder applications);
//   * several right-hand sides of the refinement share one solver launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "driver.h"
#include "kernels.h"

namespace mmd {


// MMD_DEBUG=1 in the environment prints a per-level trace to stderr.
static bool debug_on() {
  static const bool v = [] {
    const char* e = getenv("MMD_DEBUG");
    return e && e[0] && e[0] != '0';
  }();
  return v;
}

struct Workspace {
  std::map<std::string, std::pair<void*, size_t>> bufs;
  int nsm = 0;
  unsigned* bar = nullptr;  // [0] count, [1] gen
  int* status = nullptr;
  double* red = nullptr;
  int64_t* it_out = nullptr;
  int64_t* in_out = nullptr;
  int* conv = nullptr;
  // concurrent tiles of one multi-column solve: side streams and fork / join events
  cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[4] = {nullptr, nullptr, nullptr, nullptr};
  // the wide multi-column launch captured in CUDA graphs, each with the
  // arguments it was captured for (the refinement alternates between two
  // buffer sets), replayed while they are unchanged; the oldest is replaced
  static constexpr int kWideGraphs = 4;
  cudaGraphExec_t wide_exec[kWideGraphs] = {};
  WideArgs wide_key[kWideGraphs] = {};
  int wide_next = 0;
  bool wide_graph_off = false;  // capture failed once: launch directly from then on
  cudaStream_t cap = nullptr;   // private stream the graphs are recorded on (capture runs nothing)
  ~Workspace() {
    if (cap) cudaStreamDestroy(cap);
    for (auto& e : wide_exec)
      if (e) cudaGraphExecDestroy(e);
    for (int l = 0; l < 4; ++l) {
      if (side[l]) cudaStreamDestroy(side[l]);
      if (join[l]) cudaEventDestroy(join[l]);
    }
    if (fork) cudaEventDestroy(fork);
    for (auto& b : bufs) cudaFree(b.second.first);
    cudaFree(bar);
    cudaFree(status);
    cudaFree(red);
    cudaFree(it_out);
    cudaFree(in_out);
    cudaFree(conv);
  }
};

void free_workspace(mmd_handle* h) {
  delete h->ws;
  h->ws = nullptr;
}

namespace {

struct CudaFail {
  int code;
};

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x);           \
      throw CudaFail{MMD_ECUDA};                                                       \
    }                                                                                  \
  } while (0)

template <typename T>
T* buf(Workspace* ws, const std::string& name, size_t n) {
  auto it = ws->bufs.find(name);
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  if (it != ws->bufs.end() && it->second.second >= bytes) return (T*)it->second.first;
  if (it != ws->bufs.end()) {
    cudaFree(it->second.first);
    ws->bufs.erase(it);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes for " + name + " failed");
    throw CudaFail{MMD_ENOMEM};
  }
  ws->bufs[name] = {p, bytes};
  return (T*)p;
}

Workspace* get_ws(mmd_handle* h) {
  if (h->ws) return h->ws;
  Workspace* ws = new Workspace();
  cudaDeviceProp pr;
  CK(cudaGetDeviceProperties(&pr, h->device));
  ws->nsm = pr.multiProcessorCount;
  CK(cudaMalloc(&ws->bar, 64 * sizeof(unsigned)));
  CK(cudaMemset(ws->bar, 0, 64 * sizeof(unsigned)));
  CK(cudaMalloc(&ws->status, sizeof(int)));
  CK(cudaMemset(ws->status, 0, sizeof(int)));
  CK(cudaMalloc(&ws->red, sizeof(double) * 4 * 8 * 512));
  CK(cudaMalloc(&ws->it_out, sizeof(int64_t) * 8));
  CK(cudaMalloc(&ws->in_out, sizeof(int64_t)));
  CK(cudaMalloc(&ws->conv, sizeof(int) * 8));
  h->ws = ws;
  return ws;
}

Sell sell_of(const DCSR& A) {
  Sell s;
  s.nrows = A.nrows;
  s.nslices = A.nslices;
  s.ptr = A.s_ptr;
  s.len = A.s_len;
  s.row = A.s_row;
  s.col = A.s_col;
  s.val = A.s_val;
  s.val32 = A.s_val32;
  s.val2 = reinterpret_cast<const float2*>(A.s_val2);
  s.variant = A.spmv_variant;
  return s;
}

// CSR view for the V-cycle, with the lanes per row g that minimise the
// dependent load rounds a block runs on a grid of `blocks` 1024-thread blocks:
// SELL (g = 0, one row per lane): ceil(slices per block / 32 warps) x
// ceil(row length / 2); CSR with g lanes per row: ceil(rows per block /
// (1024 / g) groups) x (1 + ceil(row length / g)).  Long rows on few rows (the
// coarse Galerkin matrices, Psi^T) share a row; level 0 keeps one row per lane.
Csr32 csr32_of(const DCSR& A, int blocks) {
  Csr32 c;
  c.rowptr = A.rowptr;
  c.col = A.col;
  c.val = A.val32;
  c.nrows = A.nrows;
  const double L = std::max(1.0, A.mean_row), B = std::max(1, blocks);
  const double rows_blk = std::ceil(double(A.nrows) / B), slices_blk = std::ceil(double(A.nslices) / B);
  double best = std::ceil(slices_blk / 32.0) * std::ceil(L / 2.0);
  c.g = 0;
  for (int g : {8, 32}) {
    const double cost = std::ceil(rows_blk / (1024.0 / g)) * (1.0 + std::ceil(L / g));
    if (cost < best) {
      best = cost;
      c.g = g;
    }
  }
  return c;
}

// ------------------------------------------------------------ context
struct Ctx {
  mmd_handle* h;
  Workspace* ws;
  cudaStream_t st;
  mmd_eig_opts o;
  mmd_eig_stats S;
  double timeout_ns;

  Ctx(mmd_handle* hh, cudaStream_t s, const mmd_eig_opts& oo) : h(hh), ws(get_ws(hh)), st(s), o(oo) {
    std::memset(&S, 0, sizeof(S));
    timeout_ns = o.timeout_s * 1e9;
  }

  void sync() { CK(cudaStreamSynchronize(st)); }
  void check_status() {
    int s = 0;
    CK(cudaMemcpyAsync(&s, ws->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    sync();
    if (s == DEV_TIMEOUT) {
      set_error("a device-side grid barrier exceeded its time limit");
      throw CudaFail{MMD_ETIMEOUT};
    }
    if (s == DEV_NOTSPD) {
      set_error("a CG/PCG or Cholesky step found a non-positive pivot (matrix not SPD)");
      throw CudaFail{MMD_ENOTSPD};
    }
    if (s == DEV_NOCONV) {
      set_error("the tridiagonal QL iteration did not converge within its sweep limit");
      throw CudaFail{MMD_ENOCONV};
    }
  }
  void after_launch() {
    CK(cudaGetLastError());
    ++S.kernel_launches;
  }

  // y = A^(k) x or M^(k) x (device order), m columns of ld n
  void spmv(int k, int which, const double* x, double* y, int m) {
    const DLevel& L = h->dl[k];
    if (which == 1 && k == 0) {
      k_copy(y, x, L.n * m, st);
      after_launch();
      return;
    }
    const DCSR& A = which ? L.M : L.A;
    k_spmv(sell_of(A), x, L.n, y, L.n, m, st);
    after_launch();
  }
  void dots(const double* x, const double* y, int64_t n, int m, double* out_dev) {
    double* sc = buf<double>(ws, "dots", size_t(512) * std::max(m, 1));
    k_dots(x, y, n, n, m, out_dev, sc, st);
    S.kernel_launches += 2;
  }
  std::vector<double> dots_host(const double* x, const double* y, int64_t n, int m) {
    double* d = buf<double>(ws, "dotsout", std::max(m, 1));
    dots(x, y, n, m, d);
    std::vector<double> r(m);
    CK(cudaMemcpyAsync(r.data(), d, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    sync();
    return r;
  }

  // ---- the persistent solver
  // mode 0: CG on A_k; 1: flexible PCG with M_k; 2: CG on P A_k P (patches of level k+1)
  // B: rhs (n x m, ld n); X: initial guess (x0 = 1) / solution.  In the mixed
  // modes the FP32 solver runs inside FP64 iterative refinement (MMD_MIXED:
  // levels k >= 1, whose conditioning the decomposition bounds; MMD_MIXED_ALL:
  // level 0 too).
  void solve(int k, int mode, const double* B, double* X, int m, int x0, double tol, int maxit,
             std::vector<int64_t>* iters, int64_t* inner_total, int* notconv) {
    if (o.precision == MMD_MIXED && k == 0 && mode == 0 && h->dl[0].A.s_val2) {
      solve_df(B, X, m, x0, tol, maxit, iters, inner_total, notconv);
      return;
    }
    if ((o.precision == MMD_MIXED && k >= 1) || o.precision == MMD_MIXED_ALL) {
      solve_mixed(k, mode, B, X, m, x0, tol, maxit, iters, inner_total, notconv);
      return;
    }
    solve_raw(k, mode, false, B, X, m, x0, tol, maxit, iters, inner_total, notconv);
  }

  // Level-0 CG on A in double-float arithmetic (FP32 pairs, the matrix's
  // pair copy), checked against the FP64 residual b - A x before a column
  // is accepted; columns it leaves unconverged continue in FP64 CG from
  // their current x.
  bool use_df = false;
  // m >= 8 columns: all of them in one launch of the wide kernel per slice of
  // up to kWideMaxCols columns (row-major pair vectors, coalesced row gathers)
  void solve_wide(const double* B, double* X, int m, int x0, double tol, int maxit, std::vector<int64_t>& its,
                  std::vector<int>& cv) {
    const DLevel& L = h->dl[0];
    const int64_t n = L.n;
    const int grid = wide_max_grid(ws->nsm);
    if (grid < 1) {
      set_error("the wide solver kernel cannot be made resident");
      throw CudaFail{MMD_ECUDA};
    }
    its.assign(m, 0);
    cv.assign(m, 0);
    for (int c0 = 0; c0 < m; c0 += kWideMaxCols) {
      const int mc = std::min(kWideMaxCols, m - c0);
      WideArgs a;
      std::memset(&a, 0, sizeof(a));
      a.n = n;
      a.m = mc;
      a.ld = n;
      a.rowptr = L.A.rowptr;
      a.col = L.A.col;
      a.val2 = reinterpret_cast<const float2*>(L.A.val2);
      a.val = L.A.val;
      a.b = B + size_t(c0) * n;
      a.x = X + size_t(c0) * n;
      a.x0 = x0;
      const size_t nm = size_t(n) * mc;
      a.r = buf<double>(ws, "wd_r", nm);
      a.p = buf<double>(ws, "wd_p", nm);
      a.s = buf<double>(ws, "wd_s", nm);
      a.w = buf<double>(ws, "wd_w", nm);
      a.xd = buf<double>(ws, "wd_x", nm);
      a.q64 = buf<double>(ws, "wd_q", nm);
      a.red = buf<double>(ws, "wd_red", size_t(2) * mc * grid);
      a.red64 = buf<double>(ws, "wd_red64", size_t(2) * mc * grid);
      a.tol = tol;
      a.maxit = maxit;
      a.it_out = buf<int64_t>(ws, "wd_it", mc);
      a.conv = buf<int>(ws, "wd_cv", mc);
      unsigned* bar = buf<unsigned>(ws, "wd_bar", 64);
      a.bar.count = bar;
      a.bar.gen = bar + 32;
      a.bar.status = ws->status;
      a.bar.timeout_ns = (long long)timeout_ns;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (o.profile) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
      }
      wide_launch(a, grid, bar);
      if (o.profile) CK(cudaEventRecord(e1, st));
      CK(cudaMemcpyAsync(its.data() + c0, a.it_out, sizeof(int64_t) * mc, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(cv.data() + c0, a.conv, sizeof(int) * mc, cudaMemcpyDeviceToHost, st));
      check_status();
      if (o.profile) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int64_t itsum = 0, itmax = 0;
        for (int c = c0; c < c0 + mc; ++c) {
          itsum += its[c];
          itmax = std::max(itmax, its[c]);
        }
        const double zA = (double)L.A.nnz, nn = (double)n;
        S.pcg_launches += 1;
        S.pcg_ms += ms;
        S.pcg_bytes += itmax * (12.0 * zA + 4.0 * nn) + itsum * 72.0 * nn;
        S.pcg_flops += (double)itsum * (2.0 * zA + 10.0 * nn);
      }
    }
  }

  // The barrier reset and the wide launch as one CUDA graph: recorded on a
  // private stream at the first call with a given argument set (the
  // refinement reuses its buffers from iteration to iteration), launched on
  // the caller's stream then and replayed afterwards; if capture is refused
  // the two are issued directly from then on.
  void wide_launch(const WideArgs& a, int grid, unsigned* bar) {
    if (!ws->wide_graph_off) {
      for (int i = 0; i < Workspace::kWideGraphs; ++i)
        if (ws->wide_exec[i] && std::memcmp(&ws->wide_key[i], &a, sizeof(WideArgs)) == 0) {
          CK(cudaGraphLaunch(ws->wide_exec[i], st));
          ++S.kernel_launches;
          ++S.graph_replays;
          return;
        }
      const int slot = ws->wide_next;
      ws->wide_next = (slot + 1) % Workspace::kWideGraphs;
      if (ws->wide_exec[slot]) {
        cudaGraphExecDestroy(ws->wide_exec[slot]);
        ws->wide_exec[slot] = nullptr;
      }
      cudaGraph_t g = nullptr;
      if (!ws->cap) CK(cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking));
      bool ok = cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool issued = cudaMemsetAsync(bar, 0, sizeof(unsigned) * 64, ws->cap) == cudaSuccess &&
                            launch_wide_cg(a, grid, ws->cap) == cudaSuccess;
        ok = (cudaStreamEndCapture(ws->cap, &g) == cudaSuccess) && issued && g;
      }
      cudaGraphExec_t ex = nullptr;
      if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (ok) {
        ws->wide_exec[slot] = ex;
        std::memcpy(&ws->wide_key[slot], &a, sizeof(WideArgs));
        CK(cudaGraphLaunch(ex, st));
        ++S.kernel_launches;
        return;
      }
      ws->wide_graph_off = true;
    }
    CK(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 64, st));
    CK(launch_wide_cg(a, grid, st));
    after_launch();
  }

  void solve_df(const double* B, double* X, int m, int x0, double tol, int maxit, std::vector<int64_t>* iters,
                int64_t* inner_total, int* notconv) {
    std::vector<int64_t> its;
    std::vector<int> cv;
    if (m >= 8 && h->dl[0].A.val2) {
      solve_wide(B, X, m, x0, tol, maxit, its, cv);
    } else {
      use_df = true;
      solve_raw(0, 0, false, B, X, m, x0, tol, maxit, &its, inner_total, nullptr, nullptr, nullptr, &cv);
      use_df = false;
    }
    const int64_t n = h->dl[0].n;
    for (int c = 0; c < m; ++c) {
      if (!cv[c]) {
        std::vector<int64_t> its64;
        solve_raw(0, 0, false, B + size_t(c) * n, X + size_t(c) * n, 1, 1, tol, maxit, &its64, inner_total,
                  notconv);
        its[c] += its64[0];
        S.fp64_finishes += 1;
      }
      if (iters) iters->push_back(its[c]);
    }
  }

  // FP64 iterative refinement: R = B - A X in FP64, FP32 solve A D = R to a
  // relative tolerance no tighter than 1e-5, X += D; until ||R|| <= tol ||B||.
  void solve_mixed(int k, int mode, const double* B, double* X, int m, int x0, double tol, int maxit,
                   std::vector<int64_t>* iters, int64_t* inner_total, int* notconv) {
    if (mode == 0) {  // level-0 CG: FP32 recurrences with FP64 reliable updates, one launch
      std::vector<int64_t> its;
      std::vector<int> cv;
      solve_raw(k, 0, true, nullptr, nullptr, m, x0, tol, maxit, &its, inner_total, nullptr, B, X, &cv);
      // columns FP32 could not finish continue in FP64 CG from their current X
      const int64_t n = h->dl[k].n;
      for (int c = 0; c < m; ++c) {
        if (!cv[c]) {
          std::vector<int64_t> its64;
          solve_raw(k, 0, false, B + size_t(c) * n, X + size_t(c) * n, 1, 1, tol, maxit, &its64, inner_total,
                    notconv);
          its[c] += its64[0];
          S.fp64_finishes += 1;
        }
        if (iters) iters->push_back(its[c]);
      }
      return;
    }
    const DLevel& L = h->dl[k];
    const int64_t n = L.n;
    double* R = buf<double>(ws, "mx_R", size_t(n) * m);
    double* Y = buf<double>(ws, "mx_Y", size_t(n) * m);
    float* B32 = buf<float>(ws, "mx_B32", size_t(n) * m);
    float* D32 = buf<float>(ws, "mx_D32", size_t(n) * m);
    if (!x0) {
      k_fill(X, n * m, 0.0, st);
      after_launch();
    }
    std::vector<double> bn = dots_host(B, B, n, m);
    for (auto& v : bn) v = std::sqrt(std::max(v, 0.0));
    std::vector<int64_t> itsum(m, 0);
    bool done = false;
    for (int ref = 0; ref < 12; ++ref) {
      spmv(k, 0, X, Y, m);
      k_sub(R, B, Y, n * m, st);
      after_launch();
      if (mode == 2) {
        k_project(R, n, m, L.seg_ptr, L.phi_next, L.nseg, st);
        after_launch();
      }
      std::vector<double> rn = dots_host(R, R, n, m);
      double need = 1.0;
      bool all = true;
      for (int c = 0; c < m; ++c) {
        rn[c] = std::sqrt(std::max(rn[c], 0.0));
        if (rn[c] <= tol * bn[c] || bn[c] == 0.0) {
          k_fill(R + size_t(c) * n, n, 0.0, st);  // converged column: zero rhs, no work
          after_launch();
        } else {
          all = false;
          need = std::min(need, tol * bn[c] / rn[c]);
        }
      }
      if (all) {
        done = true;
        break;
      }
      const double tin = std::min(0.5, std::max(1e-5, 0.5 * need));
      k_to_f32(B32, R, n * m, st);
      after_launch();
      std::vector<int64_t> its;
      solve_raw(k, mode, true, B32, D32, m, 0, tin, maxit, &its, inner_total, nullptr);
      for (int c = 0; c < m; ++c) itsum[c] += its[c];
      k_add_f32(X, D32, n * m, st);
      after_launch();
    }
    if (iters)
      for (int c = 0; c < m; ++c) iters->push_back(itsum[c]);
    if (!done && notconv) ++*notconv;
  }

  // The V-cycle's level table (device memory) and work vectors, for tiles of
  // up to four columns (level 0 of the handle; mode 3 of the solver).
  void set_mg(SolverArgs& a, int deg, int only, int lane = 0) {
    const int K = (int)h->levels.size();
    const int MTmax = 4;
    std::vector<MGLevel> lv(K);
    for (int k = 0; k < K; ++k) {
      const DLevel& L = h->dl[k];
      MGLevel& g = lv[k];
      g.A = sell_of(L.A);
      g.P = sell_of(h->dl[k + 1].psi);
      g.PT = sell_of(h->dl[k + 1].psiT);
      g.cA = csr32_of(L.A, ws->nsm);
      g.cP = csr32_of(h->dl[k + 1].psi, ws->nsm);
      g.cPT = csr32_of(h->dl[k + 1].psiT, ws->nsm);
      g.dinv = L.dinv32;
      g.hi = L.gersh;
      // Chebyshev iteration on [hi / 30, hi]: theta, delta the interval's centre and
      // half-width, sigma = theta / delta, rho_0 = 1 / sigma, rho_s = 1 / (2 sigma - rho_{s-1});
      // step 0: d = D^{-1} res / theta; step s: d = rho_s rho_{s-1} d + (2 rho_s / delta) D^{-1} res
      {
        const double hi = L.gersh, lo = hi / 30.0, th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sg = th / de;
        double rho = 1.0 / sg;
        g.c1[0] = 0.f;
        g.c2[0] = (float)(1.0 / th);
        for (int st = 1; st < 8; ++st) {
          const double rn = 1.0 / (2.0 * sg - rho);
          g.c1[st] = (float)(rn * rho);
          g.c2[st] = (float)(2.0 * rn / de);
          rho = rn;
        }
      }
      g.n = L.n;
      const std::string t = std::to_string(k) + "_" + std::to_string(lane);
      g.r = buf<float>(ws, "mg_r" + t, size_t(L.n) * MTmax);
      g.x = buf<float>(ws, "mg_x" + t, size_t(L.n) * MTmax);
      g.x2 = buf<float>(ws, "mg_y" + t, size_t(L.n) * MTmax);
      g.d = buf<float>(ws, "mg_d" + t, size_t(L.n) * MTmax);
    }
    MGLevel* dlv = buf<MGLevel>(ws, "mg_levels" + std::to_string(lane), K);
    CK(cudaMemcpyAsync(dlv, lv.data(), sizeof(MGLevel) * K, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // lv is a host stack array: complete the copy before it goes
    const int64_t nK = h->dl[K].n;
    a.mg = dlv;
    a.mg_K = K;
    a.mg_deg = deg;
    a.mg_kinv = h->dl[K].kinv32;
    a.mg_rK = buf<float>(ws, "mg_rK" + std::to_string(lane), size_t(nK) * MTmax);
    a.mg_xK = buf<float>(ws, "mg_xK" + std::to_string(lane), size_t(nK) * MTmax);
    a.mg_nK = nK;
    a.mg_only = only;
  }
  int mg_deg = 2, mg_only = 0;
  int force_grid = 0;  // the autotuner's trial grid (0: tuned or heuristic)

  // The polynomial preconditioner of level 0 (mode 4): Chebyshev coefficients
  // of degree deg on [hi / poly_ratio, hi] (hi: Gershgorin bound of D^{-1} A)
  // and FP32 work vectors for tiles of up to four columns.
  void set_poly(SolverArgs& a, int deg, int lane = 0) {
    const DLevel& L = h->dl[0];
    PolyPrec& P = a.poly;
    P.deg = deg;
    const double hi = L.gersh, lo = hi / o.poly_ratio, th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sg = th / de;
    double rho = 1.0 / sg;
    P.c1[0] = 0.f;
    P.c2[0] = (float)(1.0 / th);
    for (int st = 1; st < 32; ++st) {
      const double rn = 1.0 / (2.0 * sg - rho);
      P.c1[st] = (float)(rn * rho);
      P.c2[st] = (float)(2.0 * rn / de);
      rho = rn;
    }
    P.dinv = L.dinv32;
    P.cA = csr32_of(L.A, ws->nsm);
    const int MTmax = 4;
    const std::string t = "_" + std::to_string(lane);
    P.r = buf<float>(ws, "pl_r" + t, size_t(L.n) * MTmax);
    P.x = buf<float>(ws, "pl_x" + t, size_t(L.n) * MTmax);
    P.x2 = buf<float>(ws, "pl_y" + t, size_t(L.n) * MTmax);
    P.d = buf<float>(ws, "pl_d" + t, size_t(L.n) * MTmax);
    a.mg_only = mg_only;
  }
  int poly_deg = 0;

  // Tiles of MT columns distributed round-robin over `lanes` side streams,
  // each lane with its own vectors, reduction partials, barrier counter and
  // result slots; the caller's stream forks to and joins the lanes by events.
  void solve_lanes(int k, int mode, bool fp32, const void* B, void* X, int m, int x0, double tol, int maxit,
                   std::vector<int64_t>* iters, int64_t* inner_total, int* notconv, const double* B64, double* X64,
                   std::vector<int>* conv_out, int MT, int grid, int lanes) {
    const DLevel& L = h->dl[k];
    const int64_t n = L.n;
    const size_t eb = fp32 ? sizeof(float) : sizeof(double);
    const std::string pre = fp32 ? "sv32_" : "sv_";
    if (!ws->fork) {
      CK(cudaEventCreateWithFlags(&ws->fork, cudaEventDisableTiming));
      for (int l = 0; l < 4; ++l) {
        CK(cudaStreamCreateWithFlags(&ws->side[l], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ws->join[l], cudaEventDisableTiming));
      }
    }
    const int ntiles = (m + MT - 1) / MT;
    int64_t* it_all = buf<int64_t>(ws, "ln_it", m);
    int* cv_all = buf<int>(ws, "ln_cv", m);
    int64_t* inn_all = buf<int64_t>(ws, "ln_inn", lanes);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (o.profile) {
      CK(cudaEventCreate(&t0));
      CK(cudaEventCreate(&t1));
      CK(cudaEventRecord(t0, st));
    }
    CK(cudaMemsetAsync(inn_all, 0, sizeof(int64_t) * lanes, st));
    CK(cudaEventRecord(ws->fork, st));
    for (int l = 0; l < lanes; ++l) CK(cudaStreamWaitEvent(ws->side[l], ws->fork, 0));
    for (int t = 0; t < ntiles; ++t) {
      const int l = t % lanes, c0 = t * MT, mc = std::min(MT, m - c0);
      cudaStream_t sl = ws->side[l];
      const std::string ls = "_l" + std::to_string(l);
      SolverArgs a;
      std::memset(&a, 0, sizeof(a));
      a.mode = mode;
      a.n = n;
      a.A = sell_of(L.A);
      if (mode == 1) a.M = sell_of(L.M);
      if (mode == 2) {
        a.seg_ptr = L.seg_ptr;
        a.phi = L.phi_next;
        a.nseg = L.nseg;
      }
      a.m = mc;
      a.ld = n;
      a.b = B ? (const char*)B + size_t(c0) * n * eb : nullptr;
      a.x = X ? (char*)X + size_t(c0) * n * eb : nullptr;
      a.b64 = B64 ? B64 + size_t(c0) * n : nullptr;
      a.x64 = X64 ? X64 + size_t(c0) * n : nullptr;
      a.x0 = x0;
      a.r = buf<char>(ws, pre + "r" + ls, size_t(n) * MT * eb);
      a.p = buf<char>(ws, pre + "p" + ls, size_t(n) * MT * eb);
      a.q = buf<char>(ws, pre + "q" + ls, size_t(n) * MT * eb);
      a.z = buf<char>(ws, pre + "z" + ls, size_t(n) * MT * eb);
      a.ir = buf<char>(ws, pre + "ir" + ls, size_t(n) * MT * eb);
      a.ip = buf<char>(ws, pre + "ip" + ls, size_t(n) * MT * eb);
      a.iq = buf<char>(ws, pre + "iq" + ls, size_t(n) * MT * eb);
      a.fp32 = fp32 ? 1 : 0;
      a.df = (use_df && mode == 0 && !fp32) ? 1 : 0;
      a.tol = tol;
      a.itol = 0.1 * tol;
      a.maxit = maxit;
      a.imaxit = std::min(maxit, 1000);
      a.red = buf<double>(ws, "red" + ls, size_t(4) * 8 * 512);
      a.it_out = it_all + c0;
      a.in_out = inn_all + l;
      a.conv = cv_all + c0;
      unsigned* bar = buf<unsigned>(ws, "bar" + ls, 64);
      a.bar.count = bar;
      a.bar.gen = bar + 32;
      a.bar.status = ws->status;
      a.bar.timeout_ns = (long long)timeout_ns;
      if (mode == 3) set_mg(a, mg_deg, mg_only, l);
      if (mode == 4) set_poly(a, poly_deg, l);
      CK(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 64, sl));
      CK(launch_solver(a, MT, grid, sl));
      after_launch();
    }
    for (int l = 0; l < lanes; ++l) {
      CK(cudaEventRecord(ws->join[l], ws->side[l]));
      CK(cudaStreamWaitEvent(st, ws->join[l], 0));
    }
    if (o.profile) CK(cudaEventRecord(t1, st));
    std::vector<int64_t> its(m), inn(lanes);
    std::vector<int> cv(m);
    CK(cudaMemcpyAsync(its.data(), it_all, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(cv.data(), cv_all, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(inn.data(), inn_all, sizeof(int64_t) * lanes, cudaMemcpyDeviceToHost, st));
    check_status();
    double bytes = 0, flops = 0;
    const double zA = (double)L.A.nnz, nn = (double)n;
    const double mb = fp32 ? 8.0 : 12.0, vb = fp32 ? 4.0 : 8.0;
    for (int t = 0; t < ntiles; ++t) {
      const int c0 = t * MT, mc = std::min(MT, m - c0);
      int64_t itmax = 0, itsum = 0;
      for (int c = c0; c < c0 + mc; ++c) {
        if (iters) iters->push_back(its[c]);
        if (conv_out) conv_out->push_back(cv[c]);
        if (!cv[c] && notconv) ++*notconv;
        itmax = std::max(itmax, its[c]);
        itsum += its[c];
      }
      bytes += itmax * (mb * zA + 4.0 * nn) + itsum * 9.0 * vb * nn;
      flops += (double)itsum * (2.0 * zA + (mode == 2 ? 14.0 : 10.0) * nn);
    }
    int64_t inn_sum = 0;
    for (auto v : inn) inn_sum += v;
    if (mode == 1) {
      bytes += (double)inn_sum * (mb * (double)L.M.nnz / MT + 7.5 * vb * nn);
      flops += (double)inn_sum * (2.0 * (double)L.M.nnz + 10.0 * nn);
    }
    if (inner_total) *inner_total += inn_sum;
    if (o.profile) {
      // the concurrent tiles as one timed region (their launches overlap)
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, t0, t1));
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      S.pcg_launches += ntiles;
      S.pcg_ms += ms;
      S.pcg_bytes += bytes;
      S.pcg_flops += flops;
    }
  }

  void solve_raw(int k, int mode, bool fp32, const void* B, void* X, int m, int x0, double tol, int maxit,
                 std::vector<int64_t>* iters, int64_t* inner_total, int* notconv, const double* B64 = nullptr,
                 double* X64 = nullptr, std::vector<int>* conv_out = nullptr) {
    const DLevel& L = h->dl[k];
    const int64_t n = L.n;
    // tile width (columns per solver launch): four columns on 1024 threads
    // cost 12.1 us per column-iteration on a 200k-row level-0 matrix against
    // 12.5 for eight on 512 threads, and a tile runs until its slowest column
    // is done
    const int MT = (m > 1) ? 4 : 1;
    // one block per 1024 rows (at least 16, at most one per SM): small levels
    // leave SMs free for other solves running concurrently on other streams
    const int tuned = L.grid[MT == 1 ? 0 : 1];
    int grid = std::min(solver_max_grid(MT, ws->nsm),
                        force_grid > 0 ? force_grid : tuned > 0 ? tuned : std::max(16, (int)((n + 1023) / 1024)));
    if (coop_grid_cap() > 0) grid = std::min(grid, coop_grid_cap());
    if (grid < 1) {
      set_error("solver kernel cannot be made resident");
      throw CudaFail{MMD_ECUDA};
    }
    const size_t eb = fp32 ? sizeof(float) : sizeof(double);
    const std::string pre = fp32 ? "sv32_" : "sv_";
    void* r = buf<char>(ws, pre + "r", size_t(n) * MT * eb);
    void* p = buf<char>(ws, pre + "p", size_t(n) * MT * eb);
    void* q = buf<char>(ws, pre + "q", size_t(n) * MT * eb);
    void* z = buf<char>(ws, pre + "z", size_t(n) * MT * eb);
    void* ir = buf<char>(ws, pre + "ir", size_t(n) * MT * eb);
    void* ip = buf<char>(ws, pre + "ip", size_t(n) * MT * eb);
    void* iq = buf<char>(ws, pre + "iq", size_t(n) * MT * eb);
    const int ntiles = (m + MT - 1) / MT;
    // several tiles: run them on up to four side streams at once, each grid on
    // a quarter of the SMs (a tile's iteration is latency- and barrier-bound,
    // so concurrent tiles overlap those waits); not inside the batched path,
    // whose problems already share the SMs
    const int lanes = (ntiles > 1 && coop_grid_cap() <= 0) ? std::min(ntiles, 4) : 1;
    if (lanes > 1) {
      solve_lanes(k, mode, fp32, B, X, m, x0, tol, maxit, iters, inner_total, notconv, B64, X64, conv_out, MT,
                  std::max(1, std::min(grid, ws->nsm / lanes)), lanes);
      return;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    for (int c0 = 0; c0 < m; c0 += MT) {
      const int mc = std::min(MT, m - c0);
      SolverArgs a;
      std::memset(&a, 0, sizeof(a));
      a.mode = mode;
      a.n = n;
      a.A = sell_of(L.A);
      if (mode == 1) a.M = sell_of(L.M);
      if (mode == 2) {
        a.seg_ptr = L.seg_ptr;
        a.phi = L.phi_next;
        a.nseg = L.nseg;
      }
      a.m = mc;
      a.ld = n;
      a.b = B ? (const char*)B + size_t(c0) * n * eb : nullptr;
      a.x = X ? (char*)X + size_t(c0) * n * eb : nullptr;
      a.b64 = B64 ? B64 + size_t(c0) * n : nullptr;
      a.x64 = X64 ? X64 + size_t(c0) * n : nullptr;
      a.x0 = x0;
      a.r = r;
      a.p = p;
      a.q = q;
      a.z = z;
      a.ir = ir;
      a.ip = ip;
      a.iq = iq;
      a.fp32 = fp32 ? 1 : 0;
      a.df = (use_df && mode == 0 && !fp32) ? 1 : 0;
      a.tol = tol;
      a.itol = 0.1 * tol;
      a.maxit = maxit;
      a.imaxit = std::min(maxit, 1000);
      a.red = ws->red;
      a.it_out = ws->it_out;
      a.in_out = ws->in_out;
      a.conv = ws->conv;
      a.bar.count = ws->bar;
      a.bar.gen = ws->bar + 32;
      a.bar.status = ws->status;
      a.bar.timeout_ns = (long long)timeout_ns;
      if (mode == 3) set_mg(a, mg_deg, mg_only);
      if (mode == 4) set_poly(a, poly_deg);
      CK(cudaMemsetAsync(ws->in_out, 0, sizeof(int64_t), st));
      CK(cudaMemsetAsync(ws->bar, 0, sizeof(unsigned), st));
      if (o.profile) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
      }
      CK(launch_solver(a, MT, grid, st));
      after_launch();
      if (o.profile) CK(cudaEventRecord(e1, st));
      int64_t its[8], inn = 0;
      int cv[8];
      CK(cudaMemcpyAsync(its, ws->it_out, sizeof(int64_t) * mc, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&inn, ws->in_out, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(cv, ws->conv, sizeof(int) * mc, cudaMemcpyDeviceToHost, st));
      check_status();
      int64_t itmax = 0, itsum = 0;
      for (int c = 0; c < mc; ++c) {
        if (iters) iters->push_back(its[c]);
        if (conv_out) conv_out->push_back(cv[c]);
        if (!cv[c] && notconv) ++*notconv;
        itmax = std::max(itmax, its[c]);
        itsum += its[c];
      }
      if (inner_total) *inner_total += inn;
      if (o.profile) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        S.pcg_launches += 1;
        S.pcg_ms += ms;
        // algorithmic bytes: matrix once per iteration, vectors per active column
        const double zA = (double)L.A.nnz, nn = (double)n;
        const double mb = fp32 ? 8.0 : 12.0, vb = fp32 ? 4.0 : 8.0;
        double bytes = itmax * (mb * zA + 4.0 * nn) + itsum * 9.0 * vb * nn;
        if (mode == 1) {
          const double zM = (double)L.M.nnz;
          bytes += (double)inn * (mb * zM / std::max(mc, 1) + 7.5 * vb * nn);
        }
        S.pcg_bytes += bytes;
        // algorithmic flops: per column-iteration one SpMV (2 nnz) and the
        // CG vector work (two dot products, three axpy: 10 n); mode 2 adds
        // the segment projection (4 n); per inner iteration the same on M
        double flops = (double)itsum * (2.0 * zA + (mode == 2 ? 14.0 : 10.0) * nn);
        if (mode == 1) flops += (double)inn * (2.0 * (double)L.M.nnz + 10.0 * nn);
        S.pcg_flops += flops;
      }
    }
  }

  // ---- Operator OP on level k: y = pcg(A, M x, M, 0, tol); returns iterations
  int64_t op(int k, const double* x, double* y, double tol) {
    const DLevel& L = h->dl[k];
    double* b = buf<double>(ws, "op_b", L.n);
    spmv(k, 1, x, b, 1);
    std::vector<int64_t> its;
    int64_t inner = 0;
    int nc = 0;
    const int64_t l0 = S.pcg_launches;
    const double ms0 = S.pcg_ms, by0 = S.pcg_bytes, fl0 = S.pcg_flops;
    if (k == 0 && o.poly_op > 0 && h->dl[0].dinv32) {
      // A^{-1} x by FP64 PCG preconditioned by a Chebyshev polynomial in D^{-1} A
      poly_deg = o.poly_op;
      mg_only = 0;
      solve_raw(0, 4, false, b, y, 1, 0, tol, o.max_cg_iter, &its, &inner, &nc);
    } else if (k == 0 && h->mg_ok && o.mg_op > 0 && o.method == MMD_HIERARCHICAL) {
      // A^{-1} x by FP64 PCG preconditioned by the decomposition's V-cycle
      mg_deg = o.mg_op;
      mg_only = 0;
      solve_raw(0, 3, false, b, y, 1, 0, tol, o.max_cg_iter, &its, &inner, &nc);
    } else {
      solve(k, k == 0 ? 0 : 1, b, y, 1, 0, tol, o.max_cg_iter, &its, &inner, &nc);
    }
    S.op_calls += 1;
    S.pcg_iters += its[0];
    if (k < 16) S.max_pcg_iters[k] = std::max(S.max_pcg_iters[k], its[0]);
    if (k == 0) {
      S.op0_launches += S.pcg_launches - l0;
      S.op0_ms += S.pcg_ms - ms0;
      S.op0_bytes += S.pcg_bytes - by0;
      S.op0_flops += S.pcg_flops - fl0;
      S.op0_iters += its[0];
    }
    S.inner_iters += inner;
    S.not_converged += nc;
    S.nc_solve += nc;
    return its[0];
  }
};

// Symmetric eigen-decomposition of S (m x m, destroyed) by parallel Jacobi;
// eigenvalues sorted descending (host) and eigenvectors in that order (P).
void sym_eig_desc(Ctx& c, double* S, int m, std::vector<double>& w, double* P) {
  double* V = buf<double>(c.ws, "je_V", size_t(m) * m);
  double* wk = buf<double>(c.ws, "je_w", m + 8);
  int* iw = buf<int>(c.ws, "je_i", 64);
  int* pd = buf<int>(c.ws, "je_p", m);
  GridBarrier bar;
  bar.count = c.ws->bar;
  bar.gen = c.ws->bar + 32;
  bar.status = c.ws->status;
  bar.timeout_ns = (long long)c.timeout_ns;
  CK(k_syev_jacobi(S, m, V, wk, iw, bar, c.st));
  c.after_launch();
  std::vector<double> d(m);
  CK(cudaMemcpy2DAsync(d.data(), sizeof(double), S, sizeof(double) * (m + 1), sizeof(double), m,
                       cudaMemcpyDeviceToHost, c.st));
  c.check_status();
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] > d[b]; });
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = d[ord[i]];
  CK(cudaMemcpyAsync(pd, ord.data(), sizeof(int) * m, cudaMemcpyHostToDevice, c.st));
  k_permute_cols(V, m, m, pd, m, P, m, c.st);
  c.after_launch();
}

// ------------------------------------------------------------ M-Lanczos (Algorithm 3)
struct Lanczos {
  Ctx& c;
  int k;         // level
  int64_t n;
  double* BAS;   // n x cap: [V_ini | V]
  int m0, cap;
  int j = 0;
  std::vector<double> alpha, beta;
  double* f;     // residual vector
  double wnorm = -1;
  uint64_t stream;
  int steps = 0;

  Lanczos(Ctx& cc, int kk, double* bas, int mm0, int ccap, double* ff, uint64_t s)
      : c(cc), k(kk), n(cc.h->dl[kk].n), BAS(bas), m0(mm0), cap(ccap), f(ff), stream(s) {}

  double* V() { return BAS + size_t(m0) * n; }

  // f <- f - B (B^T M f), twice (CGS2 in the M inner product) against ncols columns
  void orth(double* x, int ncols) {
    if (ncols <= 0) return;
    double* u = buf<double>(c.ws, "lz_u", n);
    double* hh = buf<double>(c.ws, "lz_h", ncols);
    double* sc = buf<double>(c.ws, "lz_sc", size_t((n + 2047) / 2048) * ncols + 64);
    for (int pass = 0; pass < 2; ++pass) {
      c.spmv(k, 1, x, u, 1);
      k_gemv_t(BAS, n, n, ncols, u, hh, sc, c.st);
      k_gemv_n(BAS, n, n, ncols, hh, -1.0, x, c.st);
      c.S.kernel_launches += 3;
    }
  }
  double mnorm(const double* x) {
    double* u = buf<double>(c.ws, "lz_u", n);
    c.spmv(k, 1, x, u, 1);
    const double v = c.dots_host(x, u, n, 1)[0];
    return std::sqrt(std::max(v, 0.0));
  }
  void random_f() {
    k_random(f, n, c.o.seed, stream, c.h->dl[k].d_perm, c.st);
    c.after_launch();
    ++stream;
    orth(f, m0 + j);
  }

  void step(double pcg_tol, double breakdown) {
    double bta = mnorm(f);
    double coupling = bta;
    if (wnorm >= 0 && bta < breakdown * wnorm) {
      random_f();
      bta = mnorm(f);
      coupling = 0.0;
    }
    if (j > 0) beta.push_back(coupling);
    double* v = V() + size_t(j) * n;
    k_copy(v, f, n, c.st);
    k_scal(v, n, 1.0 / bta, c.st);
    c.S.kernel_launches += 2;
    ++j;
    double* w = buf<double>(c.ws, "lz_w", n);
    c.op(k, v, w, pcg_tol);
    // h = B^T M w ; f = w - B h ; second pass
    const int nc = m0 + j;
    double* u = buf<double>(c.ws, "lz_u", n);
    double* hh = buf<double>(c.ws, "lz_h", nc);
    double* h2 = buf<double>(c.ws, "lz_h2", nc);
    double* sc = buf<double>(c.ws, "lz_sc", size_t((n + 2047) / 2048) * nc + 64);
    c.spmv(k, 1, w, u, 1);
    const double wn2 = c.dots_host(w, u, n, 1)[0];
    wnorm = std::sqrt(std::max(wn2, 0.0));
    k_gemv_t(BAS, n, n, nc, u, hh, sc, c.st);
    k_copy(f, w, n, c.st);
    k_gemv_n(BAS, n, n, nc, hh, -1.0, f, c.st);
    c.spmv(k, 1, f, u, 1);
    k_gemv_t(BAS, n, n, nc, u, h2, sc, c.st);
    k_gemv_n(BAS, n, n, nc, h2, -1.0, f, c.st);
    c.S.kernel_launches += 5;
    double a1 = 0, a2 = 0;
    CK(cudaMemcpyAsync(&a1, hh + nc - 1, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CK(cudaMemcpyAsync(&a2, h2 + nc - 1, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    alpha.push_back(a1 + a2);
    ++steps;
    c.S.lanczos_steps += 1;
  }

  // eigen-decomposition of T_j on the device: theta ascending (host); Y (j x j)
  // full eigenvectors and / or zl (j) their last row, by implicit QR; with
  // neither, eigenvalues only by bisection.
  void tri_eig(int jj, std::vector<double>& theta, double* Y, double* zl) {
    double* dd = buf<double>(c.ws, "te_d", jj);
    double* ee = buf<double>(c.ws, "te_e", std::max(jj - 1, 1));
    double* w = buf<double>(c.ws, "te_w", jj);
    CK(cudaMemcpyAsync(dd, alpha.data(), sizeof(double) * jj, cudaMemcpyHostToDevice, c.st));
    if (jj > 1) CK(cudaMemcpyAsync(ee, beta.data(), sizeof(double) * (jj - 1), cudaMemcpyHostToDevice, c.st));
    if (Y || zl) {
      k_tri_ql(dd, ee, jj, w, Y, jj, zl, c.ws->status, c.st);
      c.S.kernel_launches += 1;
    } else {
      k_tri_eigvals(dd, ee, jj, w, c.st);
      c.S.kernel_launches += 2;
    }
    theta.resize(jj);
    CK(cudaMemcpyAsync(theta.data(), w, sizeof(double) * jj, cudaMemcpyDeviceToHost, c.st));
    c.check_status();
  }

  // Ritz values (ascending) and residual estimates ||f||_M |e_j^T y_i|
  void ritz(std::vector<double>& theta, std::vector<double>& res) {
    double* zl = buf<double>(c.ws, "te_zl", j);
    tri_eig(j, theta, nullptr, zl);
    std::vector<double> last(j);
    CK(cudaMemcpyAsync(last.data(), zl, sizeof(double) * j, cudaMemcpyDeviceToHost, c.st));
    const double fn = mnorm(f);
    res.resize(j);
    for (int i = 0; i < j; ++i) res[i] = fn * std::fabs(last[i]);
  }

  // Algorithm 2 on a factorisation of kk + p columns: p exact shifts, keep kk
  void restart(int kk, int p) {
    const int nn = kk + p;
    std::vector<double> th;
    tri_eig(nn, th, nullptr, nullptr);
    double* dd = buf<double>(c.ws, "rs_d", nn);
    double* ee = buf<double>(c.ws, "rs_e", nn);
    double* sh = buf<double>(c.ws, "rs_sh", p);
    double* Q = buf<double>(c.ws, "rs_Q", size_t(nn) * nn);
    CK(cudaMemcpyAsync(dd, alpha.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(ee, beta.data(), sizeof(double) * (nn - 1), cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(sh, th.data(), sizeof(double) * p, cudaMemcpyHostToDevice, c.st));
    k_tri_qr_sweeps(dd, ee, nn, sh, p, Q, nn, c.st);
    c.S.kernel_launches += 2;
    std::vector<double> d2(nn), e2(nn - 1);
    double qlast = 0;
    CK(cudaMemcpyAsync(d2.data(), dd, sizeof(double) * nn, cudaMemcpyDeviceToHost, c.st));
    CK(cudaMemcpyAsync(e2.data(), ee, sizeof(double) * (nn - 1), cudaMemcpyDeviceToHost, c.st));
    CK(cudaMemcpyAsync(&qlast, Q + (nn - 1) + size_t(kk - 1) * nn, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    // f <- V_old Q(:, kk) T+(kk, kk-1) + f Q(nn-1, kk-1)
    k_scal(f, n, qlast, c.st);
    k_gemv_n(V(), n, n, nn, Q + size_t(kk) * nn, e2[kk - 1], f, c.st);
    // V <- V_old Q(:, :kk)
    double* T = buf<double>(c.ws, "rs_T", size_t(n) * kk);
    k_gemm_nn(n, kk, nn, 1.0, V(), n, Q, nn, 0.0, T, n, c.st);
    CK(cudaMemcpyAsync(V(), T, sizeof(double) * size_t(n) * kk, cudaMemcpyDeviceToDevice, c.st));
    c.S.kernel_launches += 3;
    alpha.assign(d2.begin(), d2.begin() + kk);
    beta.assign(e2.begin(), e2.begin() + (kk - 1));
    j = kk;
    wnorm = -1;
    c.S.restarts += 1;
  }
};

// ------------------------------------------------------------ Algorithm 4
struct ExtendOut {
  int m;  // total columns in BAS after extension (= m0 + new)
  std::vector<double> D;
};

// BAS: n x cap, columns [0, m0) hold V_ini on entry; on exit [0, m) hold V_ex.
ExtendOut extend(Ctx& c, int k, double* BAS, int m0, int cap, const std::vector<double>& Dini, double pcg_tol,
                 bool relative, double eps_abs, double tol_rel, bool has_mu_ex, double mu_ex, int d, int m_tar,
                 uint64_t stream0) {
  ExtendOut out{m0, Dini};
  const int64_t n = c.h->dl[k].n;
  if (m0 >= m_tar || n - m0 <= 0) return out;
  // no extension threshold (level 0, the last level computed): the searching
  // step only serves the test of mu-hat against mu_ex (Section 6), so one
  // extension goes straight to the target
  if (!has_mu_ex && c.o.d == 0) d = std::max(1, m_tar - m0);
  double* f = buf<double>(c.ws, "ex_f", n);
  Lanczos lz(c, k, BAS, m0, cap, f, stream0 + 1);
  k_random(f, n, c.o.seed, stream0, c.h->dl[k].d_perm, c.st);
  c.after_launch();
  lz.orth(f, m0);
  const int room = (int)std::min<int64_t>(n - m0, cap - m0);
  const double breakdown = 1e-10;
  // Lanczos residual test over the Ritz pairs th[skip..] (th ascending): the
  // search loop leaves out its buffer of the d smallest Ritz values (the ones
  // mu-hat is read from, refined by the next extension); the final loop,
  // whose Schur vectors are the output, tests every pair
  auto res_ok = [&](const std::vector<double>& th, const std::vector<double>& res, size_t skip) {
    for (size_t i = skip; i < th.size(); ++i) {
      const double lim = relative ? tol_rel * std::fabs(th[i]) : eps_abs;
      if (!(res[i] <= lim)) return false;
    }
    return true;
  };
  auto converge = [&](int pp, int skip) {
    for (int it = 0; it < c.o.max_restarts; ++it) {
      std::vector<double> th, res;
      lz.ritz(th, res);
      if (debug_on()) {
        double worst = 0;
        for (size_t i = skip; i < th.size(); ++i)
          worst = std::max(worst, res[i] / (relative ? tol_rel * std::fabs(th[i]) : eps_abs));
        fprintf(stderr, "[mmd] level %d converge j=%d worst res/limit=%.3e theta=[%.6e..%.6e]\n", k, lz.j, worst,
                th.front(), th.back());
      }
      if (res_ok(th, res, (size_t)skip)) return;
      const int pe = std::min(std::max(pp, lz.j), room - lz.j);
      if (pe <= 0) return;
      const int kk = lz.j;
      for (int s = 0; s < pe; ++s) lz.step(pcg_tol, breakdown);
      lz.restart(kk, pe);
    }
    c.S.not_converged += 1;
    c.S.nc_restart += 1;
  };
  const int p = std::max(1, c.o.c_r * d);
  while (true) {
    const int steps = std::min(d, room - lz.j);
    for (int s = 0; s < steps; ++s) lz.step(pcg_tol, breakdown);
    converge(p, std::min(d, lz.j - 1));
    std::vector<double> th;
    lz.tri_eig(lz.j, th, nullptr, nullptr);
    const double mu_hat = th[std::min(d, lz.j) - 1];
    if ((has_mu_ex && mu_hat < mu_ex) || lz.j >= m_tar - m0 || lz.j >= room) break;
  }
  const int m_new = lz.j;
  converge(std::max(1, c.o.c_r * m_new), 0);
  // Schur form of T: V_ex = [V_ini, V P], eigenvalues descending
  std::vector<double> th;
  double* Y = buf<double>(c.ws, "te_Y", size_t(lz.j) * lz.j);
  lz.tri_eig(lz.j, th, Y, nullptr);
  const int jn = lz.j;
  double* P = buf<double>(c.ws, "ex_P", size_t(jn) * jn);
  for (int i = 0; i < jn; ++i)  // reverse column order -> descending
    CK(cudaMemcpyAsync(P + size_t(i) * jn, Y + size_t(jn - 1 - i) * jn, sizeof(double) * jn,
                       cudaMemcpyDeviceToDevice, c.st));
  double* T = buf<double>(c.ws, "rs_T", size_t(n) * jn);
  k_gemm_nn(n, jn, jn, 1.0, lz.V(), n, P, jn, 0.0, T, n, c.st);
  CK(cudaMemcpyAsync(lz.V(), T, sizeof(double) * size_t(n) * jn, cudaMemcpyDeviceToDevice, c.st));
  c.S.kernel_launches += 1;
  out.m = m0 + jn;
  if (debug_on()) fprintf(stderr, "[mmd] level %d extend m0=%d new=%d steps=%d\n", k, m0, jn, lz.steps);
  for (int i = jn - 1; i >= 0; --i) out.D.push_back(th[i]);
  return out;
}

// ------------------------------------------------------------ M-QR, CholQR2
void mqr(Ctx& c, int k, const double* F, double* Q, int m) {
  const int64_t n = c.h->dl[k].n;
  double* MQ = buf<double>(c.ws, "qr_MQ", size_t(n) * m);
  double* G = buf<double>(c.ws, "qr_G", size_t(m) * m);
  double* Ri = buf<double>(c.ws, "qr_Ri", size_t(m) * m);
  double* T = buf<double>(c.ws, "qr_T", size_t(n) * m);
  double* s = buf<double>(c.ws, "qr_s", m);
  const size_t gsl = std::max<size_t>(size_t(8) << 20, size_t(m) * m * 4);
  double* gs = buf<double>(c.ws, "gemm_scratch", gsl);
  c.spmv(k, 1, F, MQ, m);
  std::vector<double> nr = c.dots_host(F, MQ, n, m);
  for (auto& x : nr) x = 1.0 / std::sqrt(std::max(x, 1e-300));
  CK(cudaMemcpyAsync(s, nr.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.st));
  CK(cudaMemcpyAsync(Q, F, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
  k_scale_cols(Q, n, n, m, s, c.st);
  c.after_launch();
  for (int pass = 0; pass < 2; ++pass) {
    c.spmv(k, 1, Q, MQ, m);
    k_gemm_tn(m, m, n, 1.0, Q, n, MQ, n, 0.0, G, m, gs, gsl, c.st);
    k_symmetrise(G, m, m, c.st);
    k_potrf_upper(G, m, m, c.ws->status, c.st);
    k_trinv_upper(G, m, m, Ri, m, c.st);
    k_gemm_nn(n, m, m, 1.0, Q, n, Ri, m, 0.0, T, n, c.st);
    CK(cudaMemcpyAsync(Q, T, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
    c.S.kernel_launches += 6;
  }
  c.check_status();
}

// ------------------------------------------------------------ Algorithm 5
// Q0 (n_k x m, device order of level k) and D (descending mu) from level k+1.
// On exit Qout holds the first mh refined columns and D is resized to mh.
int refine(Ctx& c, int k, double* Q0, std::vector<double>& D, double tol_rel, double mu_re, double eps_h,
           double delta_h, double* Qout) {
  const int m = (int)D.size();
  if (m == 0) return 0;
  const auto t_start = std::chrono::steady_clock::now();
  const DLevel& L = c.h->dl[k];
  const int64_t n = L.n;
  double* R = buf<double>(c.ws, "rf_R", size_t(n) * m);
  double* G = buf<double>(c.ws, "rf_G", size_t(n) * m);
  double* F = buf<double>(c.ws, "rf_F", size_t(n) * m);
  double* Q = buf<double>(c.ws, "rf_Q", size_t(n) * m);
  double* W = buf<double>(c.ws, "rf_W", size_t(n) * m);
  double* Qp = buf<double>(c.ws, "rf_Qp", size_t(n) * m);
  double* T1 = buf<double>(c.ws, "rf_T1", size_t(n) * m);
  double* Dd = buf<double>(c.ws, "rf_D", m);
  double* Sm = buf<double>(c.ws, "rf_S", size_t(m) * m);
  double* P = buf<double>(c.ws, "rf_P", size_t(m) * m);
  double* X = buf<double>(c.ws, "rf_X", size_t(m) * m);
  const size_t gsl = std::max<size_t>(size_t(8) << 20, size_t(m) * m * 4);
  double* gs = buf<double>(c.ws, "gemm_scratch", gsl);
  // g_i = CG(B, U^T M q_i): in coordinates U g, rhs = P M q_i
  c.spmv(k, 1, Q0, R, m);
  k_project(R, n, m, L.seg_ptr, L.phi_next, L.nseg, c.st);
  c.after_launch();
  {
    std::vector<int64_t> its;
    int nc = 0;
    c.solve(k, 2, R, G, m, 0, tol_rel, c.o.max_cg_iter, &its, nullptr, &nc);
    c.S.b_calls += m;
    for (auto t : its) c.S.b_iters += t;
    c.S.not_converged += nc;
    c.S.nc_solve += nc;
  }
  // F0 = Q0 D + U G
  CK(cudaMemcpyAsync(Dd, D.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.st));
  CK(cudaMemcpyAsync(F, Q0, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
  k_scale_cols(F, n, n, m, Dd, c.st);
  k_axpy(F, G, n * m, 1.0, c.st);
  CK(cudaMemcpyAsync(Qp, Q0, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
  c.S.kernel_launches += 2;
  const double stop = tol_rel / std::sqrt(1.0 + eps_h * delta_h);
  int mh = m;
  bool done = false;
  for (int it = 1; it <= c.o.max_refine_iter; ++it) {
    mqr(c, k, F, Q, m);
    c.spmv(k, 1, Q, W, m);
    // F = pcg(A, W, M, D Q, tol)
    CK(cudaMemcpyAsync(Dd, D.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(F, Q, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
    k_scale_cols(F, n, n, m, Dd, c.st);
    c.after_launch();
    {
      std::vector<int64_t> its;
      int64_t inner = 0;
      int nc = 0;
      if (k == 0 && c.o.poly_refine > 0 && c.h->dl[0].dinv32) {
        // warm-started level-0 solves preconditioned by a Chebyshev polynomial (FP32, FP64 PCG)
        c.poly_deg = c.o.poly_refine;
        c.mg_only = 0;
        c.solve_raw(0, 4, false, W, F, m, 1, tol_rel, c.o.max_cg_iter, &its, &inner, &nc);
      } else if (k == 0 && c.h->mg_ok && c.o.mg_refine > 0) {
        // warm-started level-0 solves preconditioned by the decomposition (FP32 V-cycle, FP64 PCG)
        c.mg_deg = c.o.mg_refine;
        c.mg_only = 0;
        c.solve_raw(0, 3, false, W, F, m, 1, tol_rel, c.o.max_cg_iter, &its, &inner, &nc);
      } else {
        c.solve(k, k == 0 ? 0 : 1, W, F, m, 1, tol_rel, c.o.max_cg_iter, &its, &inner, &nc);
      }
      c.S.refine_pcg_calls += m;
      for (auto t : its) {
        c.S.refine_pcg_iters += t;
        if (k < 16) c.S.max_pcg_iters[k] = std::max(c.S.max_pcg_iters[k], t);
      }
      c.S.inner_iters += inner;
      c.S.not_converged += nc;
      c.S.nc_solve += nc;
    }
    // S = W^T F, eig descending (parallel Jacobi)
    k_gemm_tn(m, m, n, 1.0, W, n, F, n, 0.0, Sm, m, gs, gsl, c.st);
    k_symmetrise(Sm, m, m, c.st);
    c.S.kernel_launches += 3;
    std::vector<double> w;
    sym_eig_desc(c, Sm, m, w, P);
    for (int i = 0; i < m; ++i) D[i] = w[i];
    // renew m_h: mu_mh >= mu_re, and a gap to the end of the window
    // (mu_mh >= mu_ml alpha / (1 + beta), efficiency condition (ii) of Section 6)
    const double thr = std::max(mu_re, D[m - 1] * c.o.alpha / (1.0 + c.o.beta));
    mh = 0;
    while (mh < m && D[mh] >= thr) ++mh;
    // Q <- Q P, F <- F P, MQ = W P
    k_gemm_nn(n, m, m, 1.0, Q, n, P, m, 0.0, T1, n, c.st);
    std::swap(Q, T1);
    k_gemm_nn(n, m, m, 1.0, F, n, P, m, 0.0, T1, n, c.st);
    std::swap(F, T1);
    k_gemm_nn(n, m, m, 1.0, W, n, P, m, 0.0, T1, n, c.st);  // T1 = M Q_new
    c.S.kernel_launches += 3;
    c.S.refine_iters += 1;
    double dq = 0;
    if (mh > 0) {
      k_gemm_tn(mh, mh, n, 1.0, Qp, n, T1, n, 0.0, X, mh, gs, gsl, c.st);
      // W <- Q_mh - Qp_mh X  (W is free now)
      CK(cudaMemcpyAsync(W, Q, sizeof(double) * size_t(n) * mh, cudaMemcpyDeviceToDevice, c.st));
      k_gemm_nn(n, mh, mh, -1.0, Qp, n, X, mh, 1.0, W, n, c.st);
      c.S.kernel_launches += 2;
      std::vector<double> nr = c.dots_host(W, W, n * (int64_t)mh, 1);
      dq = std::sqrt(std::max(nr[0], 0.0));
    }
    CK(cudaMemcpyAsync(Qp, Q, sizeof(double) * size_t(n) * m, cudaMemcpyDeviceToDevice, c.st));
    if (dq < stop) {
      done = true;
      break;
    }
  }
  if (!done) {
    c.S.not_converged += 1;
    c.S.nc_refine += 1;
  }
  CK(cudaMemcpyAsync(Qout, Q, sizeof(double) * size_t(n) * mh, cudaMemcpyDeviceToDevice, c.st));
  D.resize(mh);
  if (debug_on()) {
    c.sync();
    fprintf(stderr, "[mmd] level %d refine m=%d mh=%d done=%d time %.1f ms\n", k, m, mh, (int)done,
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count());
  }
  return mh;
}

// ------------------------------------------------------------ coarsest level
// Generalized eigenproblem A z = lambda M z (M = I when K = 0); returns mu
// descending and Z (device, n x n, M-orthonormal columns in that order).
void coarsest(Ctx& c, int K, std::vector<double>& mu, double* Zout) {
  const DLevel& L = c.h->dl[K];
  const int n = (int)L.n;
  double* Ad = buf<double>(c.ws, "co_A", size_t(n) * n);
  double* Md = buf<double>(c.ws, "co_M", size_t(n) * n);
  double* Tt = buf<double>(c.ws, "co_T", size_t(n) * n);
  double* Y = buf<double>(c.ws, "co_Y", size_t(n) * n);
  k_csr_to_dense(L.A.rowptr, L.A.col, L.A.val, n, Ad, n, c.st);
  c.after_launch();
  if (K > 0) {
    k_csr_to_dense(L.M.rowptr, L.M.col, L.M.val, n, Md, n, c.st);
    k_potrf_lower(Md, n, n, c.ws->status, c.st);
    k_trsm_llnn(Md, n, n, Ad, n, n, c.st);   // L^{-1} A
    k_transpose_sq(Ad, n, n, Tt, n, c.st);   // (L^{-1} A)^T = A L^{-T}
    k_trsm_llnn(Md, n, n, Tt, n, n, c.st);   // L^{-1} A L^{-T}
    k_symmetrise(Tt, n, n, c.st);
    c.S.kernel_launches += 6;
  } else {
    CK(cudaMemcpyAsync(Tt, Ad, sizeof(double) * size_t(n) * n, cudaMemcpyDeviceToDevice, c.st));
  }
  // eigenvalues of C = L^{-1} A L^{-T}; Jacobi sorted descending in lambda, so
  // reverse to ascending lambda = descending mu
  std::vector<double> wd;
  sym_eig_desc(c, Tt, n, wd, Tt == Y ? nullptr : Y);
  std::vector<int> rev(n);
  for (int i = 0; i < n; ++i) rev[i] = n - 1 - i;
  int* pd = buf<int>(c.ws, "co_rev", n);
  CK(cudaMemcpyAsync(pd, rev.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c.st));
  k_permute_cols(Y, n, n, pd, n, Ad, n, c.st);  // Ad <- Y reversed (A no longer needed)
  c.after_launch();
  if (K > 0) {
    k_trsm_lltn(Md, n, n, Ad, n, n, c.st);  // z = L^{-T} y
    c.after_launch();
  }
  c.check_status();
  mu.resize(n);
  for (int i = 0; i < n; ++i) mu[i] = 1.0 / wd[n - 1 - i];
  Y = Ad;
  CK(cudaMemcpyAsync(Zout, Y, sizeof(double) * size_t(n) * n, cudaMemcpyDeviceToDevice, c.st));
}

}  // namespace

// ------------------------------------------------------------ entry points
int level_spmv(mmd_handle* h, int k, int which, const double* x, double* y, cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    Ctx c(h, st, o);
    const DLevel& L = h->dl[k];
    double* a = buf<double>(c.ws, "ls_a", L.n);
    double* b = buf<double>(c.ws, "ls_b", L.n);
    k_gather(x, L.n, L.d_perm, L.n, 1, a, L.n, st);
    c.spmv(k, which, a, b, 1);
    k_scatter(b, L.n, L.d_perm, L.n, 1, y, L.n, st);
    c.sync();
    CK(cudaGetLastError());
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

// reps back-to-back SpMVs on device-order vectors between two events on the
// stream: the kernel's own time, without the permutations and the
// synchronisation of level_spmv.
int level_spmv_timed(mmd_handle* h, int k, int which, const double* x, double* y, int reps, float* ms,
                     cudaStream_t st) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    Ctx c(h, st, o);
    const DLevel& L = h->dl[k];
    double* a = buf<double>(c.ws, "lt_a", L.n);
    double* b = buf<double>(c.ws, "lt_b", L.n);
    k_gather(x, L.n, L.d_perm, L.n, 1, a, L.n, st);
    c.spmv(k, which, a, b, 1);  // warm-up
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) c.spmv(k, which, a, b, 1);
    CK(cudaEventRecord(e1, st));
    k_scatter(b, L.n, L.d_perm, L.n, 1, y, L.n, st);
    c.sync();
    CK(cudaGetLastError());
    float t = 0;
    CK(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / reps;
  } catch (const CudaFail& f) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return f.code;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MMD_OK;
}

int level_op(mmd_handle* h, int k, const double* x, double* y, double tol, int max_iter, int64_t* iters,
             cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    o.max_cg_iter = max_iter;
    Ctx c(h, st, o);
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const DLevel& L = h->dl[k];
    double* a = buf<double>(c.ws, "ls_a", L.n);
    double* b = buf<double>(c.ws, "ls_b", L.n);
    k_gather(x, L.n, L.d_perm, L.n, 1, a, L.n, st);
    const int64_t it = c.op(k, a, b, tol);
    k_scatter(b, L.n, L.d_perm, L.n, 1, y, L.n, st);
    c.sync();
    CK(cudaGetLastError());
    if (iters) *iters = it;
    if (c.S.not_converged) {
      set_error("mmd_level_op: PCG reached max_iter");
      return MMD_ENOCONV;
    }
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

// Y = OP(X) for m columns: the multi-right-hand-side solve of the refinement
// (Algorithm 5) on caller vectors, in tiles of 4 columns per launch.
int level_op_block(mmd_handle* h, int k, int m, const double* x, double* y, double tol, int max_iter,
                   int64_t* iters, int precision, cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    o.max_cg_iter = max_iter;
    o.precision = precision;
    Ctx c(h, st, o);
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const DLevel& L = h->dl[k];
    double* a = buf<double>(c.ws, "lb_a", size_t(L.n) * m);
    double* b = buf<double>(c.ws, "lb_b", size_t(L.n) * m);
    double* z = buf<double>(c.ws, "lb_z", size_t(L.n) * m);
    k_gather(x, L.n, L.d_perm, L.n, m, a, L.n, st);
    c.spmv(k, 1, a, b, m);
    std::vector<int64_t> its;
    int64_t inner = 0;
    int nc = 0;
    c.solve(k, k == 0 ? 0 : 1, b, z, m, 0, tol, max_iter, &its, &inner, &nc);
    k_scatter(z, L.n, L.d_perm, L.n, m, y, L.n, st);
    c.sync();
    CK(cudaGetLastError());
    if (iters)
      for (int i = 0; i < m; ++i) iters[i] = its[i];
    if (nc) {
      set_error("mmd_level_op_block: PCG reached max_iter");
      return MMD_ENOCONV;
    }
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

// The solver autotuner: for every level that runs CG / PCG solves (k < K)
// and both tile widths, 20 iterations of CG on A^(k) from a random
// right-hand side (tolerance out of reach, so every trial runs the same
// iterations) are timed with events at each candidate grid that is resident
// and leaves at least 64 rows per block; the fastest grid is kept in the
// level.  Runs once per handle, on a private stream, before any solve.
int tune_solver(mmd_handle* h) {
  cudaStream_t st = nullptr;
  try {
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    Ctx c(h, st, o);
    const int K = (int)h->levels.size();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int k = 0; k < K; ++k) {
      DLevel& L = h->dl[k];
      const int64_t n = L.n;
      for (int w = 0; w < 2; ++w) {
        const int mt = w == 0 ? 1 : 4;
        double* B = buf<double>(c.ws, "tn_b", size_t(n) * mt);
        double* X = buf<double>(c.ws, "tn_x", size_t(n) * mt);
        k_random(B, n * mt, 12345u, 77u + w, nullptr, st);
        c.after_launch();
        const int gmax = solver_max_grid(mt, c.ws->nsm);
        float best = 0.f;
        int bestg = 0;
        bool warm = false;
        for (int ci = 0; ci < 8; ++ci) {
          const int g = std::min(kTuneGrids[ci], c.ws->nsm);
          L.grid_us[w][ci] = 0.f;
          if (g > gmax || (ci > 0 && int64_t(g) * 64 > n) || (ci > 0 && g == std::min(kTuneGrids[ci - 1], c.ws->nsm)))
            continue;
          c.force_grid = g;
          std::vector<int64_t> its;
          if (!warm) {  // first launch of this instance on this level: not timed
            c.solve_raw(k, 0, false, B, X, mt, 0, 1e-300, 20, &its, nullptr, nullptr);
            its.clear();
            warm = true;
          }
          CK(cudaEventRecord(e0, st));
          c.solve_raw(k, 0, false, B, X, mt, 0, 1e-300, 20, &its, nullptr, nullptr);
          CK(cudaEventRecord(e1, st));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          const float us = 1e3f * ms / 21.f;  // 20 iterations + the closing product
          L.grid_us[w][ci] = us;
          if (bestg == 0 || us < best) {
            best = us;
            bestg = g;
          }
        }
        L.grid[w] = bestg;
      }
    }
    c.force_grid = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(st));
    cudaStreamDestroy(st);
  } catch (const CudaFail& f) {
    if (st) cudaStreamDestroy(st);
    return f.code;
  }
  return MMD_OK;
}

int level_poly(mmd_handle* h, int m, const double* R, double* Z, int deg, double ratio, cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    o.poly_ratio = ratio;
    Ctx c(h, st, o);
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const DLevel& L = h->dl[0];
    double* a = buf<double>(c.ws, "lv_a", size_t(L.n) * m);
    double* b = buf<double>(c.ws, "lv_b", size_t(L.n) * m);
    k_gather(R, L.n, L.d_perm, L.n, m, a, L.n, st);
    c.poly_deg = deg;
    c.mg_only = 1;
    std::vector<int64_t> its;
    c.solve_raw(0, 4, false, a, b, m, 0, 1e-30, 1, &its, nullptr, nullptr);
    k_scatter(b, L.n, L.d_perm, L.n, m, Z, L.n, st);
    c.sync();
    CK(cudaGetLastError());
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

int level_vcycle(mmd_handle* h, int m, const double* R, double* Z, int deg, cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    Ctx c(h, st, o);
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const DLevel& L = h->dl[0];
    double* a = buf<double>(c.ws, "lv_a", size_t(L.n) * m);
    double* b = buf<double>(c.ws, "lv_b", size_t(L.n) * m);
    k_gather(R, L.n, L.d_perm, L.n, m, a, L.n, st);
    c.mg_deg = deg;
    c.mg_only = 1;
    std::vector<int64_t> its;
    c.solve_raw(0, 3, false, a, b, m, 0, 1e-30, 1, &its, nullptr, nullptr);
    k_scatter(b, L.n, L.d_perm, L.n, m, Z, L.n, st);
    c.sync();
    CK(cudaGetLastError());
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

int level_bsolve(mmd_handle* h, int k, const double* q, double* x, double tol, int max_iter, int64_t* iters,
                 cudaStream_t st) {
  try {
    mmd_eig_opts o;
    mmd_default_eig_opts(&o);
    Ctx c(h, st, o);
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const int lv = k - 1;  // level of the vectors
    const DLevel& L = h->dl[lv];
    double* a = buf<double>(c.ws, "ls_a", L.n);
    double* b = buf<double>(c.ws, "ls_b", L.n);
    double* r = buf<double>(c.ws, "ls_r", L.n);
    k_gather(q, L.n, L.d_perm, L.n, 1, a, L.n, st);
    c.spmv(lv, 1, a, r, 1);
    k_project(r, L.n, 1, L.seg_ptr, L.phi_next, L.nseg, st);
    std::vector<int64_t> its;
    int nc = 0;
    c.solve(lv, 2, r, b, 1, 0, tol, max_iter, &its, nullptr, &nc);
    k_scatter(b, L.n, L.d_perm, L.n, 1, x, L.n, st);
    c.sync();
    CK(cudaGetLastError());
    if (iters) *iters = its[0];
    if (nc) {
      set_error("mmd_level_bsolve: CG reached max_iter");
      return MMD_ENOCONV;
    }
  } catch (const CudaFail& f) {
    return f.code;
  }
  return MMD_OK;
}

// Wall time of level k's work (coarsest solve, or refinement + extension),
// Section 7's per-level computation time.
static void S_level_mark(Ctx& c, int k, std::chrono::steady_clock::time_point t0) {
  const double now = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  double prev = 0;
  for (int j = 0; j < 16; ++j) prev += c.S.t_level_ms[j];
  c.S.t_level_ms[k] = now - prev;
  if (debug_on()) fprintf(stderr, "[mmd] level %d time %.1f ms\n", k, now - prev);
}

int run_eig(mmd_handle* h, int N, double tol, const mmd_eig_opts& o, double* lambda, double* Vout, int outdev,
            mmd_eig_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)o.stream;
  int rc = MMD_OK;
  Ctx* cp = nullptr;
  try {
    cp = new Ctx(h, st, o);
    Ctx& c = *cp;
    CK(cudaMemsetAsync(c.ws->status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c.ws->bar, 0, 2 * sizeof(unsigned), st));
    const int K = (int)h->levels.size();
    const int64_t n0 = h->dl[0].n;
    // scratch of the tridiagonal kernels, sized for the largest Lanczos / Ritz matrix
    const int tri_max = std::max<int>(4 * N + 128, (int)h->dl[K].n + 8);
    {
      double* bounds = buf<double>(c.ws, "tri_bounds", 4);
      double* e2 = buf<double>(c.ws, "tri_e2", tri_max);
      int* cst = buf<int>(c.ws, "tri_cstart", tri_max + 1);
      int* ncl = buf<int>(c.ws, "tri_ncl", 1);
      double* work = buf<double>(c.ws, "tri_work", size_t(8) * tri_max * tri_max);
      int* iwork = buf<int>(c.ws, "tri_iwork", size_t(tri_max) * tri_max);
      set_tri_scratch(bounds, e2, cst, ncl, work, iwork);
    }
    if (o.stop_level > K) {
      set_error("eig_leftmost: stop_level " + std::to_string(o.stop_level) + " exceeds the handle's K = " +
                std::to_string(K));
      throw CudaFail{MMD_EINVAL};
    }
    std::vector<double> D;
    int m = 0;
    double* Vh = nullptr;
    int out_level = 0;  // the level whose coefficient vectors Vh holds at the end
    if (o.method == MMD_IRLM_CG) {
      // Section 8's baseline: no decomposition; Algorithm 4 at level 0 from an
      // empty basis with searching step d = N, so one extension reaches N
      // columns and each restart of its final loop applies N exact shifts
      // (N wanted pairs, 2N Lanczos vectors); OP is plain CG on A.
      const int64_t n = h->dl[0].n;
      const int d = N;
      const int cap = (int)std::min<int64_t>(n, 2 * ((int64_t)N + d) + 8);
      double* BAS = buf<double>(c.ws, "BAS_b", size_t(n) * cap);
      ExtendOut ex = extend(c, 0, BAS, 0, cap, std::vector<double>(), 0.1 * tol, true, 0.0, tol, false, 0.0, d, N,
                            1000);
      m = ex.m;
      D = ex.D;
      Vh = BAS;
      c.sync();
      S_level_mark(c, 0, t0);
    } else {
    // ---- coarsest level (Algorithm 6, first step)
    std::vector<double> mu;
    const int nK = (int)h->dl[K].n;
    double* Z = buf<double>(c.ws, "co_Z", size_t(nK) * nK);
    coarsest(c, K, mu, Z);
    c.S.mu1 = mu.empty() ? 0.0 : mu[0];
    const double mu1 = c.S.mu1;
    const int last = o.stop_level;  // the last level computed
    if (K == 0) {
      m = std::min(N, nK);
      D.assign(mu.begin(), mu.begin() + m);
      Vh = buf<double>(c.ws, "V_cur", size_t(n0) * m);
      CK(cudaMemcpyAsync(Vh, Z, sizeof(double) * size_t(n0) * m, cudaMemcpyDeviceToDevice, st));
    } else {
      const double epsK = h->dl[K].eps;
      int keep = 0;
      if (last == K) {
        keep = (int)mu.size();  // the coarse-level approximation: the N largest mu of the pencil
      } else {
        while (keep < (int)mu.size() && mu[keep] >= o.beta * epsK) ++keep;
      }
      m = std::min(keep, N);
      D.assign(mu.begin(), mu.begin() + m);
      Vh = buf<double>(c.ws, "V_cur", size_t(nK) * std::max(m, 1));
      if (m) CK(cudaMemcpyAsync(Vh, Z, sizeof(double) * size_t(nK) * m, cudaMemcpyDeviceToDevice, st));
      uint64_t stream = 1000;
      c.sync();
      if (K < 16) S_level_mark(c, K, t0);
      for (int k = K - 1; k >= last; --k) {
        const DLevel& L = h->dl[k];
        const int64_t n = L.n;
        const int d = o.d > 0 ? o.d : std::max(1, (int)std::min<int64_t>(n / 10, N / 10));
        const int cap = (int)std::min<int64_t>(n, (int64_t)m + 2 * (N + d) + 8);
        double* BAS = buf<double>(c.ws, k % 2 ? "BAS_a" : "BAS_b", size_t(n) * cap);
        // transfer V <- Psi^(k+1) V (Algorithm 6, coefficient reform)
        double* Q0 = buf<double>(c.ws, "Q0", size_t(n) * std::max(m, 1));
        if (m) {
          k_spmv(sell_of(h->dl[k + 1].psi), Vh, h->dl[k + 1].n, Q0, n, m, st);
          c.after_launch();
        }
        double eps_h = 0, delta_h = 0, tol_rel, eps_abs = 0;
        bool relative;
        const double eps_l = h->dl[k + 1].eps;
        if (k >= 1) {
          eps_h = L.eps;
          delta_h = L.delta;
          tol_rel = std::min(0.1, std::max(1e-14, 0.1 * eps_h / mu1));
          eps_abs = 0.1 * eps_h;
          relative = false;
        } else {
          tol_rel = tol;
          relative = true;
        }
        const double pcg_tol = (k == 0) ? 0.1 * tol_rel : tol_rel;
        const double mu_re = o.alpha * eps_l;
        // Algorithm 5: refined pairs into BAS[:, :mh]
        int mh = refine(c, k, Q0, D, pcg_tol, mu_re, eps_h, delta_h, BAS);
        // Algorithm 4; the last level computed extends to N pairs (no extension threshold)
        ExtendOut ex = extend(c, k, BAS, mh, cap, D, pcg_tol, relative, eps_abs, tol, k > last,
                              o.beta * eps_h, d, N, stream);
        stream += 1000;
        m = ex.m;
        D = ex.D;
        Vh = BAS;
        c.sync();
        if (k < 16) S_level_mark(c, k, t0);
      }
      out_level = last;
    }
    }
    // a result on level s >= 1: V = Psi^(1) ... Psi^(s) V^(s) (Algorithm 6, last line)
    for (int j = out_level; j >= 1 && m > 0; --j) {
      double* T = buf<double>(c.ws, j % 2 ? "xfer_a" : "xfer_b", size_t(h->dl[j - 1].n) * m);
      k_spmv(sell_of(h->dl[j].psi), Vh, h->dl[j].n, T, h->dl[j - 1].n, m, st);
      c.after_launch();
      Vh = T;
    }
    // ---- outputs: N largest mu -> ascending lambda, natural order, normalised
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return D[a] > D[b]; });
    const int nout = std::min(N, m);
    double* Vs = buf<double>(c.ws, "out_V", size_t(n0) * std::max(nout, 1));
    double* Vn = buf<double>(c.ws, "out_Vn", size_t(n0) * std::max(nout, 1));
    std::vector<double> lam(N, 0.0);
    for (int i = 0; i < nout; ++i) {
      CK(cudaMemcpyAsync(Vs + size_t(i) * n0, Vh + size_t(order[i]) * n0, sizeof(double) * n0,
                         cudaMemcpyDeviceToDevice, st));
      lam[i] = 1.0 / D[order[i]];
    }
    // residuals in device order (norms are permutation invariant)
    double* lamd = buf<double>(c.ws, "out_lam", std::max(nout, 1));
    double* resd = buf<double>(c.ws, "out_res", std::max(nout, 1));
    double* rsc = buf<double>(c.ws, "out_rsc", size_t(n0) * std::max(nout, 1) + size_t(512) * std::max(nout, 1));
    if (nout) {
      k_scatter(Vs, n0, h->dl[0].d_perm, n0, nout, Vn, n0, st);
      k_normalise_sign(Vn, n0, n0, nout, nullptr, st);
      k_gather(Vn, n0, h->dl[0].d_perm, n0, nout, Vs, n0, st);
      CK(cudaMemcpyAsync(lamd, lam.data(), sizeof(double) * nout, cudaMemcpyHostToDevice, st));
      k_residuals(sell_of(h->dl[0].A), n0, Vs, n0, nout, lamd, resd, rsc, st);
      c.S.kernel_launches += 3 + 4;
    }
    std::vector<double> res(nout);
    if (nout) CK(cudaMemcpyAsync(res.data(), resd, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
    c.sync();
    double mx = 0;
    int nconv = 0;
    for (int i = 0; i < nout; ++i) {
      const double r = res[i] / h->normA_inf;
      mx = std::max(mx, r);
      if (r <= tol) ++nconv;
    }
    c.S.max_rel_residual = mx;
    c.S.n_converged = nconv;
    c.S.norm_A = h->normA_inf;
    c.S.n_levels = K + 1;
    const cudaMemcpyKind kv = outdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind kl = outdev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if (nout) CK(cudaMemcpyAsync(Vout, Vn, sizeof(double) * size_t(n0) * nout, kv, st));
    // keep the result for eig_grad
    if (nout) {
      double* lv = buf<double>(c.ws, "last_V", size_t(n0) * nout);
      CK(cudaMemcpyAsync(lv, Vn, sizeof(double) * size_t(n0) * nout, cudaMemcpyDeviceToDevice, st));
    }
    h->last_lam.assign(lam.begin(), lam.begin() + nout);
    h->last_N = nout;
    if (kl == cudaMemcpyHostToHost)
      std::memcpy(lambda, lam.data(), sizeof(double) * N);
    else
      CK(cudaMemcpyAsync(lambda, lam.data(), sizeof(double) * N, kl, st));
    c.sync();
    if (nout < N || c.S.not_converged) rc = MMD_ENOCONV;
    if (nout < N) set_error("eig_leftmost: fewer pairs than requested were found");
    else if (rc) set_error("eig_leftmost: an iteration cap was reached");
  } catch (const CudaFail& f) {
    rc = f.code;
    if (h->ws) {
      cudaMemset(h->ws->bar, 0, 2 * sizeof(unsigned));
      cudaMemset(h->ws->status, 0, sizeof(int));
    }
  }
  if (cp) {
    cp->S.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = cp->S;
    delete cp;
  }
  return rc;
}

// ------------------------------------------------------------ adjoint
// dL/dval for every stored entry of the input CSR from the last eig_leftmost
// result (lambda_i, v_i), i < N, and the loss gradients gl = dL/dlambda,
// Gv = dL/dV (may be NULL):
//   U = V diag(gl) + Y,  y_i = -(A - lambda_i I)^+ g_i  (in-block terms plus
//   a CG solve of (A - lambda_i I) z = -(I - V V^T) g_i on range(I - V V^T)),
//   G_e = sum_i U(r_e, i) V(c_e, i).
int run_grad(mmd_handle* h, const double* gl_in, const double* Gv_in, int in_dev, double* out, int out_dev,
             const mmd_eig_opts& o) {
  cudaStream_t st = (cudaStream_t)o.stream;
  int rc = MMD_OK;
  try {
    Ctx c(h, st, o);
    const int N = h->last_N;
    const int64_t n = h->A0.nrows, nnz = h->A0.nnz();
    if (N < 1) {
      set_error("eig_grad: no eig_leftmost result on this handle");
      return MMD_EINVAL;
    }
    double* V = buf<double>(c.ws, "last_V", size_t(n) * N);
    double* U = buf<double>(c.ws, "gr_U", size_t(n) * N);
    double* Gv = buf<double>(c.ws, "gr_Gv", size_t(n) * N);
    double* gld = buf<double>(c.ws, "gr_gl", N);
    const cudaMemcpyKind ki = in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(gld, gl_in, sizeof(double) * N, ki, st));
    CK(cudaMemcpyAsync(U, V, sizeof(double) * size_t(n) * N, cudaMemcpyDeviceToDevice, st));
    k_scale_cols(U, n, n, N, gld, st);
    c.after_launch();
    if (Gv_in) {
      CK(cudaMemcpyAsync(Gv, Gv_in, sizeof(double) * size_t(n) * N, ki, st));
      std::vector<double> gn = c.dots_host(Gv, Gv, n, N);
      // C = V^T Gv (N x N) -> in-block coefficients D_ji = C_ji / (lambda_i - lambda_j)
      double* Cd = buf<double>(c.ws, "gr_C", size_t(N) * N);
      const size_t gsl = std::max<size_t>(size_t(8) << 20, size_t(N) * N * 4);
      double* gs = buf<double>(c.ws, "gemm_scratch", gsl);
      k_gemm_tn(N, N, n, 1.0, V, n, Gv, n, 0.0, Cd, N, gs, gsl, st);
      c.after_launch();
      std::vector<double> C(size_t(N) * N), D(size_t(N) * N, 0.0);
      CK(cudaMemcpyAsync(C.data(), Cd, sizeof(double) * N * N, cudaMemcpyDeviceToHost, st));
      c.sync();
      const std::vector<double>& lam = h->last_lam;
      for (int i = 0; i < N; ++i) {
        if (!(gn[i] > 0)) continue;
        for (int j = 0; j < N; ++j)
          if (j != i && std::fabs(lam[i] - lam[j]) > 1e-14 * std::max(std::fabs(lam[i]), 1.0))
            D[j + size_t(i) * N] = C[j + size_t(i) * N] / (lam[i] - lam[j]);
      }
      CK(cudaMemcpyAsync(Cd, D.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice, st));
      k_gemm_nn(n, N, N, 1.0, V, n, Cd, N, 1.0, U, n, st);  // U += V D
      c.after_launch();
      // complement: (A - lambda_i I) z = -(I - V V^T) g_i, CG on range(I - V V^T)
      // (natural order: the level-0 matrix is applied through gather/scatter)
      const DLevel& L0 = h->dl[0];
      double* z = buf<double>(c.ws, "gr_z", n);
      double* r = buf<double>(c.ws, "gr_r", n);
      double* p = buf<double>(c.ws, "gr_p", n);
      double* q = buf<double>(c.ws, "gr_q", n);
      double* t1 = buf<double>(c.ws, "gr_t1", n);
      double* t2 = buf<double>(c.ws, "gr_t2", n);
      double* hv = buf<double>(c.ws, "gr_h", N);
      double* sc = buf<double>(c.ws, "lz_sc", size_t((n + 2047) / 2048) * N + 64);
      auto project = [&](double* x) {
        k_gemv_t(V, n, n, N, x, hv, sc, st);
        k_gemv_n(V, n, n, N, hv, -1.0, x, st);
        c.S.kernel_launches += 3;
      };
      auto apply = [&](const double* x, double shift, double* y) {  // y = P (A - shift I) x
        k_gather(x, n, L0.d_perm, n, 1, t1, n, st);
        k_spmv(sell_of(L0.A), t1, n, t2, n, 1, st);
        k_scatter(t2, n, L0.d_perm, n, 1, y, n, st);
        k_axpy(y, x, n, -shift, st);
        c.S.kernel_launches += 4;
        project(y);
      };
      for (int i = 0; i < N; ++i) {
        if (!(gn[i] > 0)) continue;
        k_copy(r, Gv + size_t(i) * n, n, st);
        k_scal(r, n, -1.0, st);
        project(r);
        k_fill(z, n, 0.0, st);
        k_copy(p, r, n, st);
        c.S.kernel_launches += 4;
        double rr = c.dots_host(r, r, n, 1)[0];
        const double bn = std::sqrt(rr);
        for (int it = 0; it < o.max_cg_iter && std::sqrt(rr) > 1e-12 * bn && bn > 0; ++it) {
          apply(p, lam[i], q);
          const double pq = c.dots_host(p, q, n, 1)[0];
          if (!(pq > 0)) {
            set_error("eig_grad: the shifted complement operator is not positive definite "
                      "(lambda_i >= lambda_{N+1}?)");
            throw CudaFail{MMD_ENOTSPD};
          }
          const double al = rr / pq;
          k_axpy(z, p, n, al, st);
          k_axpy(r, q, n, -al, st);
          const double rn = c.dots_host(r, r, n, 1)[0];
          k_scal(p, n, rn / rr, st);
          k_axpy(p, r, n, 1.0, st);
          c.S.kernel_launches += 4;
          rr = rn;
        }
        project(z);
        k_axpy(U + size_t(i) * n, z, n, 1.0, st);
        c.after_launch();
      }
    }
    // G_e = sum_i U(r_e, i) V(c_e, i) over the input pattern
    if (!h->d_in_rowptr) {
      CK(cudaMalloc(&h->d_in_rowptr, sizeof(int32_t) * (n + 1)));
      CK(cudaMalloc(&h->d_in_col, sizeof(int32_t) * nnz));
      CK(cudaMemcpy(h->d_in_rowptr, h->A0.rowptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_in_col, h->A0.col.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    }
    double* G = out_dev ? out : buf<double>(c.ws, "gr_G", nnz);
    k_sddmm(h->d_in_rowptr, h->d_in_col, n, U, V, n, N, G, st);
    c.after_launch();
    if (!out_dev) CK(cudaMemcpyAsync(out, G, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    c.sync();
  } catch (const CudaFail& f) {
    rc = f.code;
  }
  return rc;
}

}  // namespace mmd
