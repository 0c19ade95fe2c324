// Host construction of the Multiresolution Matrix Decomposition (Section 2.3).
//
// Per level k, from A = A^(k-1) (M^(0) = I):
//   1. partition the pattern of A (diagonal excluded) into patches by a
//      two-pass integer-only aggregation;
//   2. phi_j = unit eigenvector of the smallest eigenvalue of the patch's
//      interior energy A[S,S] - diag(sum_{c not in S} |a_rc|) (Section 2.2,
//      q = 1), the closed energy A[S,S] when that is not PSD; the sign makes
//      the largest-|.| entry positive;
//   3. error factor eps = max_j 1/lambda_2 (Section 2.2) and condition factor
//      delta = max_j 1/(phi^T A[S,S]^{-1} phi) (Theorem 2.2);
//   4. normalised Householder vector u_j = (phi_j + sign(phi_j[0]) e_0)/|.|,
//      whose reflector's columns 1.. span the complement U_j (Section 2.3);
//   5. psi_j minimising psi^T A psi subject to phi_i^T psi = delta_ij for the
//      patches i inside its support Omega_j (the energy-minimising basis of
//      Section 2.2 restricted to P_j and whole neighbouring patches);
//   6. A^(k) = Psi^T A Psi and M^(k) = Psi^T M^(k-1) Psi on their symbolic
//      patterns, symmetrised.
// Small dense problems use the routines below (cyclic Jacobi, Cholesky).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "build_gpu.h"
#include "mmd_internal.h"

namespace mmd {
namespace {

// ------------------------------------------------------------ small dense
// Symmetric eigen-decomposition by the cyclic Jacobi method (Golub and Van
// Loan, Matrix Computations, Section 8.5).  a: n x n row-major, destroyed.
// w: eigenvalues ascending, v: n x n row-major, column i = eigenvector i.
void jacobi_eig(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
  v.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) v[size_t(i) * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double x = a[size_t(i) * n + j] * a[size_t(i) * n + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[size_t(p) * n + q];
        if (apq == 0.0) continue;
        double app = a[size_t(p) * n + p], aqq = a[size_t(q) * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a[size_t(k) * n + p], akq = a[size_t(k) * n + q];
          a[size_t(k) * n + p] = c * akp - s * akq;
          a[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a[size_t(p) * n + k], aqk = a[size_t(q) * n + k];
          a[size_t(p) * n + k] = c * apk - s * aqk;
          a[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[size_t(k) * n + p], vkq = v[size_t(k) * n + q];
          v[size_t(k) * n + p] = c * vkp - s * vkq;
          v[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[size_t(x) * n + x] < a[size_t(y) * n + y]; });
  w.resize(n);
  std::vector<double> vs(size_t(n) * n);
  for (int c = 0; c < n; ++c) {
    w[c] = a[size_t(idx[c]) * n + idx[c]];
    for (int r = 0; r < n; ++r) vs[size_t(r) * n + c] = v[size_t(r) * n + idx[c]];
  }
  v.swap(vs);
}

// In-place lower Cholesky of an n x n row-major SPD matrix.  Returns false if
// a pivot is not positive.
// sum_{k < len} x[k] y[k] with four independent partial sums (the row dot
// products of the Cholesky below are its whole cost; one accumulator would
// serialise on the FMA latency)
static inline double dot4(const double* x, const double* y, int len) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int k = 0;
  for (; k + 4 <= len; k += 4) {
    s0 += x[k] * y[k];
    s1 += x[k + 1] * y[k + 1];
    s2 += x[k + 2] * y[k + 2];
    s3 += x[k + 3] * y[k + 3];
  }
  for (; k < len; ++k) s0 += x[k] * y[k];
  return (s0 + s1) + (s2 + s3);
}

bool cholesky(int n, std::vector<double>& a) {
  for (int j = 0; j < n; ++j) {
    const double* aj = a.data() + size_t(j) * n;
    const double s = a[size_t(j) * n + j] - dot4(aj, aj, j);
    if (!(s > 0)) return false;
    const double d = std::sqrt(s);
    a[size_t(j) * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double* ai = a.data() + size_t(i) * n;
      ai[j] = (ai[j] - dot4(ai, aj, j)) / d;
    }
  }
  return true;
}

// Solve L L^T x = b in place (L from cholesky).
void chol_solve(int n, const std::vector<double>& L, double* b) {
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[size_t(i) * n + k] * b[k];
    b[i] = t / L[size_t(i) * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k < n; ++k) t -= L[size_t(k) * n + i] * b[k];
    b[i] = t / L[size_t(i) * n + i];
  }
}

double entry(const HCSR& A, int r, int c) {
  const int32_t* b = A.col.data() + A.rowptr[r];
  const int32_t* e = A.col.data() + A.rowptr[r + 1];
  const int32_t* p = std::lower_bound(b, e, c);
  return (p != e && *p == c) ? A.val[p - A.col.data()] : 0.0;
}

int nthreads_of(const mmd_build_opts* o) {
#ifdef _OPENMP
  return o->threads > 0 ? o->threads : omp_get_max_threads();
#else
  (void)o;
  return 1;
#endif
}

// ------------------------------------------------------------ 1. partition
void partition(const HCSR& A, int s_max, std::vector<int32_t>& patch_of, std::vector<int32_t>& patch_ptr,
               std::vector<int32_t>& patch_rows) {
  const int64_t n = A.nrows;
  std::vector<int64_t> po(n, -1);
  std::vector<int64_t> sizes;
  auto seed = [&](int64_t i) {
    int64_t pid = (int64_t)sizes.size();
    po[i] = pid;
    int64_t cnt = 1;
    for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      int32_t j = A.col[k];
      if (j == i) continue;
      if (cnt >= s_max) break;
      if (po[j] < 0) {
        po[j] = pid;
        ++cnt;
      }
    }
    sizes.push_back(cnt);
  };
  for (int64_t i = 0; i < n; ++i) {
    if (po[i] >= 0) continue;
    bool all_free = true;
    for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      int32_t j = A.col[k];
      if (j != i && po[j] >= 0) {
        all_free = false;
        break;
      }
    }
    if (all_free) seed(i);
  }
  std::vector<int64_t> nb;
  for (int64_t i = 0; i < n; ++i) {
    if (po[i] >= 0) continue;
    nb.clear();
    for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      int32_t j = A.col[k];
      if (j != i && po[j] >= 0) nb.push_back(po[j]);
    }
    std::sort(nb.begin(), nb.end());
    int64_t best = -1, bestc = 0;
    for (size_t a = 0; a < nb.size();) {
      size_t b = a;
      while (b < nb.size() && nb[b] == nb[a]) ++b;
      int64_t p = nb[a], c = int64_t(b - a);
      if (sizes[p] < 2 * s_max && c > bestc) {
        best = p;
        bestc = c;
      }
      a = b;
    }
    if (best >= 0) {
      po[i] = best;
      ++sizes[best];
    } else {
      seed(i);
    }
  }
  const int64_t np = (int64_t)sizes.size();
  patch_of.resize(n);
  patch_ptr.assign(np + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    patch_of[i] = (int32_t)po[i];
    ++patch_ptr[po[i] + 1];
  }
  for (int64_t p = 0; p < np; ++p) patch_ptr[p + 1] += patch_ptr[p];
  std::vector<int32_t> fill(patch_ptr.begin(), patch_ptr.end() - 1);
  patch_rows.resize(n);
  for (int64_t i = 0; i < n; ++i) patch_rows[fill[po[i]]++] = (int32_t)i;
}

// 1 / lambda_2 of the patch energy of rows S (ascending): interior energy
// A[S,S] - diag(sum of |a_rc| outside S), or A[S,S] when that is not PSD --
// the patch's share of eps(P) (Section 2.2).
double inv_lambda2(const HCSR& A, const std::vector<double>& rowabs, const std::vector<int32_t>& S) {
  const int s = (int)S.size();
  std::vector<double> AS(size_t(s) * s, 0.0), E, w, V;
  for (int x = 0; x < s; ++x) {
    const int r = S[x];
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      auto it = std::lower_bound(S.begin(), S.end(), A.col[k]);
      if (it != S.end() && *it == A.col[k]) AS[size_t(x) * s + (it - S.begin())] = A.val[k];
    }
  }
  E = AS;
  for (int x = 0; x < s; ++x) {
    double inside = 0;
    for (int y = 0; y < s; ++y) inside += std::fabs(AS[size_t(x) * s + y]);
    E[size_t(x) * s + x] -= rowabs[S[x]] - inside;
  }
  jacobi_eig(s, E, w, V);
  double wmax = 0;
  for (double t : w) wmax = std::max(wmax, std::fabs(t));
  if (w[0] < -1e-10 * wmax) {
    E = AS;
    jacobi_eig(s, E, w, V);
  }
  return 1.0 / w[1];
}

// Bound eps(P) by splitting weakly attached rows off their patches (build
// option peel > 0).  eps(P) is a maximum over patches, so one row hanging on
// its patch by small weights sets it for the whole level.  With cap = peel x
// the lower median of 1/lambda_2 over patches of two or more rows, each patch
// in id order loses, while 1/lambda_2 > cap, the row with the smallest
// interior weight sum_{u in S, u != v} |a_vu| (ties: lowest row); removed
// rows become singleton patches numbered after the existing ones in removal
// order.  Sums run over the CSR row in column order.
void peel_patches(const HCSR& A, double mult, std::vector<int32_t>& patch_of, std::vector<int32_t>& patch_ptr,
                  std::vector<int32_t>& patch_rows, int nthreads) {
  if (!(mult > 0)) return;
  const int64_t n = A.nrows, np = (int64_t)patch_ptr.size() - 1;
  std::vector<double> rowabs(n, 0.0);
  for (int64_t r = 0; r < n; ++r) {
    double t = 0;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) t += std::fabs(A.val[k]);
    rowabs[r] = t;
  }
  std::vector<double> inv(np, -1.0);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t j = 0; j < np; ++j) {
    if (patch_ptr[j + 1] - patch_ptr[j] < 2) continue;
    std::vector<int32_t> S(patch_rows.begin() + patch_ptr[j], patch_rows.begin() + patch_ptr[j + 1]);
    inv[j] = inv_lambda2(A, rowabs, S);
  }
  std::vector<double> sorted;
  for (double t : inv)
    if (t >= 0) sorted.push_back(t);
  if (sorted.empty()) return;
  std::sort(sorted.begin(), sorted.end());
  const double cap = mult * sorted[(sorted.size() - 1) / 2];
  // each patch is peeled independently; removals are numbered in patch order
  std::vector<std::vector<int32_t>> removed(np);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
  for (int64_t j = 0; j < np; ++j) {
    if (!(inv[j] > cap)) continue;
    std::vector<int32_t> S(patch_rows.begin() + patch_ptr[j], patch_rows.begin() + patch_ptr[j + 1]);
    while (S.size() > 1 && inv_lambda2(A, rowabs, S) > cap) {
      int32_t best = -1;
      double bw = 0;
      for (int32_t v : S) {
        double t = 0;
        for (int32_t k = A.rowptr[v]; k < A.rowptr[v + 1]; ++k) {
          const int32_t c = A.col[k];
          if (c != v && std::binary_search(S.begin(), S.end(), c)) t += std::fabs(A.val[k]);
        }
        if (best < 0 || t < bw) {
          best = v;
          bw = t;
        }
      }
      S.erase(std::find(S.begin(), S.end(), best));
      removed[j].push_back(best);
    }
  }
  int32_t nxt = (int32_t)np;
  for (int64_t j = 0; j < np; ++j)
    for (int32_t v : removed[j]) patch_of[v] = nxt++;
  const int64_t np2 = nxt;
  patch_ptr.assign(np2 + 1, 0);
  for (int64_t i = 0; i < n; ++i) ++patch_ptr[patch_of[i] + 1];
  for (int64_t p = 0; p < np2; ++p) patch_ptr[p + 1] += patch_ptr[p];
  std::vector<int32_t> fill(patch_ptr.begin(), patch_ptr.end() - 1);
  patch_rows.resize(n);
  for (int64_t i = 0; i < n; ++i) patch_rows[fill[patch_of[i]]++] = (int32_t)i;
}

// ------------------------------------------------------------ 2-4. bases
struct PatchOut {
  double eps = 0, delta = 0;
  int closed = 0;
  bool ok = true;
};

void local_bases(const HCSR& A, const std::vector<int32_t>& patch_ptr, const std::vector<int32_t>& patch_rows,
                 const std::vector<int32_t>& patch_of, std::vector<double>& phi, std::vector<double>& uhat,
                 double& eps, double& delta, int& used_closed, bool& ok, int nthreads) {
  const int64_t np = (int64_t)patch_ptr.size() - 1;
  phi.assign(A.nrows, 0.0);
  uhat.assign(A.nrows, 0.0);
  std::vector<double> rowabs(A.nrows, 0.0);
  for (int64_t r = 0; r < A.nrows; ++r) {
    double s = 0;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) s += std::fabs(A.val[k]);
    rowabs[r] = s;
  }
  std::vector<PatchOut> po(np);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t j = 0; j < np; ++j) {
    const int a = patch_ptr[j], b = patch_ptr[j + 1], s = b - a;
    std::vector<double> AS(size_t(s) * s, 0.0), E, w, V;
    std::vector<double> outside(s);
    for (int x = 0; x < s; ++x) {
      const int r = patch_rows[a + x];
      double inside = 0;
      for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
        const int c = A.col[k];
        if (patch_of[c] != j) continue;
        const int y = int(std::lower_bound(patch_rows.begin() + a, patch_rows.begin() + b, c) - (patch_rows.begin() + a));
        AS[size_t(x) * s + y] = A.val[k];
        inside += std::fabs(A.val[k]);
      }
      outside[x] = rowabs[r] - inside;
    }
    E = AS;
    for (int x = 0; x < s; ++x) E[size_t(x) * s + x] -= outside[x];
    jacobi_eig(s, E, w, V);
    double wmax = 0;
    for (double t : w) wmax = std::max(wmax, std::fabs(t));
    if (s > 1 && w[0] < -1e-10 * wmax) {  // a singleton's phi is 1 either way
      po[j].closed = 1;
      E = AS;
      jacobi_eig(s, E, w, V);
    }
    std::vector<double> p(s);
    int imax = 0;
    for (int x = 0; x < s; ++x) {
      p[x] = V[size_t(x) * s + 0];
      if (std::fabs(p[x]) > std::fabs(p[imax])) imax = x;
    }
    if (!(p[imax] > 0))
      for (double& t : p) t = -t;
    if (s > 1) po[j].eps = 1.0 / w[1];
    std::vector<double> L = AS, xs = p;
    if (!cholesky(s, L)) {
      po[j].ok = false;
      continue;
    }
    chol_solve(s, L, xs.data());
    double ptx = 0;
    for (int x = 0; x < s; ++x) ptx += p[x] * xs[x];
    po[j].delta = 1.0 / ptx;
    std::vector<double> u = p;
    u[0] += (p[0] >= 0 ? 1.0 : -1.0);
    double un = 0;
    for (double t : u) un += t * t;
    un = std::sqrt(un);
    for (int x = 0; x < s; ++x) {
      phi[a + x] = p[x];
      uhat[a + x] = u[x] / un;
    }
  }
  eps = 0;
  delta = 0;
  used_closed = 0;
  ok = true;
  for (const auto& q : po) {
    eps = std::max(eps, q.eps);
    delta = std::max(delta, q.delta);
    used_closed += q.closed;
    ok = ok && q.ok;
  }
}

// ------------------------------------------------------------ 5. Psi
void neighbourhoods(const HCSR& A, const std::vector<int32_t>& patch_of, const std::vector<int32_t>& patch_ptr,
                    const std::vector<int32_t>& patch_rows, int omega_max, int loc_radius,
                    std::vector<int32_t>& optr, std::vector<int32_t>& orows, int nthreads) {
  const int64_t np = (int64_t)patch_ptr.size() - 1;
  std::vector<std::vector<int32_t>> per(np);
  // patch adjacency (sorted, unique), for rings beyond the first
  std::vector<std::vector<int32_t>> adj;
  if (loc_radius >= 2) {
    adj.assign(np, {});
    for (int64_t r = 0; r < A.nrows; ++r)
      for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
        const int32_t pr = patch_of[r], pc = patch_of[A.col[k]];
        if (pc != pr) adj[pr].push_back(pc);
      }
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int64_t p = 0; p < np; ++p) {
      std::sort(adj[p].begin(), adj[p].end());
      adj[p].erase(std::unique(adj[p].begin(), adj[p].end()), adj[p].end());
    }
  }
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t j = 0; j < np; ++j) {
    std::vector<int32_t> chosen{(int32_t)j};
    int total = patch_ptr[j + 1] - patch_ptr[j];
    if (loc_radius >= 1) {
      std::vector<int32_t> nbp;
      for (int32_t x = patch_ptr[j]; x < patch_ptr[j + 1]; ++x) {
        const int r = patch_rows[x];
        for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
          const int c = A.col[k];
          if (c == r) continue;
          if (patch_of[c] != j) nbp.push_back(patch_of[c]);
        }
      }
      std::sort(nbp.begin(), nbp.end());
      std::vector<std::pair<int, int32_t>> ranked;  // (-count, patch)
      for (size_t a = 0; a < nbp.size();) {
        size_t b = a;
        while (b < nbp.size() && nbp[b] == nbp[a]) ++b;
        ranked.push_back({-int(b - a), nbp[a]});
        a = b;
      }
      std::sort(ranked.begin(), ranked.end());
      std::vector<int32_t> seen{(int32_t)j}, ring;
      for (const auto& t : ranked) {
        seen.push_back(t.second);
        const int sz = patch_ptr[t.second + 1] - patch_ptr[t.second];
        if (total + sz <= omega_max) {
          chosen.push_back(t.second);
          ring.push_back(t.second);
          total += sz;
        }
      }
      // ring t >= 2: patches adjacent to ring t - 1 not offered before, ascending
      for (int t = 2; t <= loc_radius; ++t) {
        std::sort(seen.begin(), seen.end());
        std::vector<int32_t> cand;
        for (int32_t p : ring)
          for (int32_t q : adj[p])
            if (!std::binary_search(seen.begin(), seen.end(), q)) cand.push_back(q);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        ring.clear();
        for (int32_t p : cand) {
          seen.push_back(p);
          const int sz = patch_ptr[p + 1] - patch_ptr[p];
          if (total + sz <= omega_max) {
            chosen.push_back(p);
            ring.push_back(p);
            total += sz;
          }
        }
      }
    }
    std::vector<int32_t> rows;
    rows.reserve(total);
    for (int32_t p : chosen)
      for (int32_t x = patch_ptr[p]; x < patch_ptr[p + 1]; ++x) rows.push_back(patch_rows[x]);
    std::sort(rows.begin(), rows.end());
    per[j].swap(rows);
  }
  optr.assign(np + 1, 0);
  for (int64_t j = 0; j < np; ++j) optr[j + 1] = optr[j] + (int32_t)per[j].size();
  orows.resize(optr[np]);
  for (int64_t j = 0; j < np; ++j) std::copy(per[j].begin(), per[j].end(), orows.begin() + optr[j]);
}

bool localized_psi(const HCSR& A, const std::vector<int32_t>& patch_of, const std::vector<double>& phi,
                   const std::vector<int32_t>& patch_rows, const std::vector<int32_t>& optr,
                   const std::vector<int32_t>& orows, int64_t np, std::vector<double>& psival, int nthreads) {
  std::vector<double> phi_of_row(A.nrows);
  for (int64_t x = 0; x < A.nrows; ++x) phi_of_row[patch_rows[x]] = phi[x];
  psival.assign(orows.size(), 0.0);
  bool ok = true;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(&& : ok)
  for (int64_t j = 0; j < np; ++j) {
    const int a = optr[j], m = optr[j + 1] - a;
    const int32_t* O = orows.data() + a;
    std::vector<double> L(size_t(m) * m, 0.0);
    for (int x = 0; x < m; ++x) {
      const int r = O[x];
      for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
        const int32_t* p = std::lower_bound(O, O + m, A.col[k]);
        if (p != O + m && *p == A.col[k]) L[size_t(x) * m + (p - O)] = A.val[k];
      }
    }
    // constraint patches inside Omega_j, ascending id
    std::vector<int32_t> plist(m);
    for (int x = 0; x < m; ++x) plist[x] = patch_of[O[x]];
    std::vector<int32_t> up = plist;
    std::sort(up.begin(), up.end());
    up.erase(std::unique(up.begin(), up.end()), up.end());
    const int nc = (int)up.size();
    if (!cholesky(m, L)) {
      ok = false;
      continue;
    }
    // Y = A_OO^{-1} C^T, columns a = constraint patch
    std::vector<double> Y(size_t(nc) * m, 0.0);  // row a = column a of Y
    for (int x = 0; x < m; ++x) {
      const int ai = int(std::lower_bound(up.begin(), up.end(), plist[x]) - up.begin());
      Y[size_t(ai) * m + x] = phi_of_row[O[x]];
    }
    std::vector<double> Cx(size_t(nc) * m);
    Cx = Y;  // C rows (phi restricted), kept for S = C Y
    // L L^T y = c for every constraint row; the backward sweep reads L^T by
    // rows (same sums, same order as chol_solve, contiguous loads)
    std::vector<double> LT(size_t(m) * m);
    for (int x = 0; x < m; ++x)
      for (int y = 0; y <= x; ++y) LT[size_t(y) * m + x] = L[size_t(x) * m + y];
    for (int ai = 0; ai < nc; ++ai) {
      double* b = Y.data() + size_t(ai) * m;
      for (int i = 0; i < m; ++i) {
        double t = b[i];
        const double* Li = L.data() + size_t(i) * m;
        for (int k = 0; k < i; ++k) t -= Li[k] * b[k];
        b[i] = t / Li[i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double t = b[i];
        const double* Ui = LT.data() + size_t(i) * m;
        for (int k = i + 1; k < m; ++k) t -= Ui[k] * b[k];
        b[i] = t / Ui[i];
      }
    }
    std::vector<double> S(size_t(nc) * nc, 0.0);
    for (int ai = 0; ai < nc; ++ai)
      for (int bi = 0; bi < nc; ++bi) {
        double t = 0;
        for (int x = 0; x < m; ++x) t += Cx[size_t(ai) * m + x] * Y[size_t(bi) * m + x];
        S[size_t(ai) * nc + bi] = t;
      }
    for (int ai = 0; ai < nc; ++ai)
      for (int bi = 0; bi < ai; ++bi) {
        double t = 0.5 * (S[size_t(ai) * nc + bi] + S[size_t(bi) * nc + ai]);
        S[size_t(ai) * nc + bi] = S[size_t(bi) * nc + ai] = t;
      }
    std::vector<double> e(nc, 0.0);
    e[std::lower_bound(up.begin(), up.end(), (int32_t)j) - up.begin()] = 1.0;
    if (!cholesky(nc, S)) {
      ok = false;
      continue;
    }
    chol_solve(nc, S, e.data());
    for (int x = 0; x < m; ++x) {
      double t = 0;
      for (int ai = 0; ai < nc; ++ai) t += Y[size_t(ai) * m + x] * e[ai];
      psival[a + x] = t;
    }
  }
  return ok;
}

// Psi as CSR (rows = fine level, cols = patches) from its column lists.
void psi_to_csr(int64_t n_fine, int64_t np, const std::vector<int32_t>& optr, const std::vector<int32_t>& orows,
                const std::vector<double>& psival, HCSR& P) {
  P.nrows = n_fine;
  P.ncols = np;
  P.rowptr.assign(n_fine + 1, 0);
  for (int32_t r : orows) ++P.rowptr[r + 1];
  for (int64_t r = 0; r < n_fine; ++r) P.rowptr[r + 1] += P.rowptr[r];
  P.col.resize(orows.size());
  P.val.resize(orows.size());
  std::vector<int32_t> fill(P.rowptr.begin(), P.rowptr.end() - 1);
  for (int64_t j = 0; j < np; ++j)  // ascending column -> sorted rows
    for (int32_t x = optr[j]; x < optr[j + 1]; ++x) {
      const int32_t r = orows[x];
      P.col[fill[r]] = (int32_t)j;
      P.val[fill[r]] = psival[x];
      ++fill[r];
    }
}

// ------------------------------------------------------------ 6. Galerkin
// C = X * Y with the symbolic pattern of the product (no pruning).
void spgemm(const HCSR& X, const HCSR& Y, HCSR& C, int nthreads) {
  C.nrows = X.nrows;
  C.ncols = Y.ncols;
  const int64_t n = X.nrows;
  std::vector<std::vector<int32_t>> cols(n);
  std::vector<std::vector<double>> vals(n);
#pragma omp parallel num_threads(nthreads)
  {
    std::vector<double> acc(Y.ncols, 0.0);
    std::vector<int32_t> mark(Y.ncols, -1);
#pragma omp for schedule(dynamic, 64)
    for (int64_t r = 0; r < n; ++r) {
      std::vector<int32_t>& cl = cols[r];
      for (int32_t k = X.rowptr[r]; k < X.rowptr[r + 1]; ++k) {
        const int32_t m = X.col[k];
        const double xv = X.val[k];
        for (int32_t q = Y.rowptr[m]; q < Y.rowptr[m + 1]; ++q) {
          const int32_t c = Y.col[q];
          if (mark[c] != r) {
            mark[c] = (int32_t)r;
            acc[c] = 0.0;
            cl.push_back(c);
          }
          acc[c] += xv * Y.val[q];
        }
      }
      std::sort(cl.begin(), cl.end());
      vals[r].resize(cl.size());
      for (size_t t = 0; t < cl.size(); ++t) vals[r][t] = acc[cl[t]];
    }
  }
  C.rowptr.assign(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) C.rowptr[r + 1] = C.rowptr[r] + (int32_t)cols[r].size();
  C.col.resize(C.rowptr[n]);
  C.val.resize(C.rowptr[n]);
  for (int64_t r = 0; r < n; ++r) {
    std::copy(cols[r].begin(), cols[r].end(), C.col.begin() + C.rowptr[r]);
    std::copy(vals[r].begin(), vals[r].end(), C.val.begin() + C.rowptr[r]);
  }
}

void transpose(const HCSR& X, HCSR& T) {
  T.nrows = X.ncols;
  T.ncols = X.nrows;
  T.rowptr.assign(X.ncols + 1, 0);
  for (int32_t c : X.col) ++T.rowptr[c + 1];
  for (int64_t r = 0; r < X.ncols; ++r) T.rowptr[r + 1] += T.rowptr[r];
  T.col.resize(X.col.size());
  T.val.resize(X.val.size());
  std::vector<int32_t> fill(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int64_t r = 0; r < X.nrows; ++r)
    for (int32_t k = X.rowptr[r]; k < X.rowptr[r + 1]; ++k) {
      const int32_t c = X.col[k];
      T.col[fill[c]] = (int32_t)r;
      T.val[fill[c]] = X.val[k];
      ++fill[c];
    }
}

void symmetrise(HCSR& C) {
  std::vector<double> v(C.val.size());
  for (int64_t r = 0; r < C.nrows; ++r)
    for (int32_t k = C.rowptr[r]; k < C.rowptr[r + 1]; ++k) v[k] = 0.5 * (C.val[k] + entry(C, C.col[k], (int)r));
  C.val.swap(v);
}

HCSR identity(int64_t n) {
  HCSR I;
  I.nrows = I.ncols = n;
  I.rowptr.resize(n + 1);
  I.col.resize(n);
  I.val.assign(n, 1.0);
  for (int64_t i = 0; i <= n; ++i) I.rowptr[i] = (int32_t)i;
  for (int64_t i = 0; i < n; ++i) I.col[i] = (int32_t)i;
  return I;
}

int validate(const mmd_csr* A) {
  if (!A || A->n < 1 || A->nnz < A->n || !A->rowptr || !A->col || !A->val) return MMD_EINVAL;
  if (A->nnz >= (int64_t(1) << 31)) return MMD_EINVAL;
  return MMD_OK;
}

}  // namespace

int build_host(const mmd_csr* Ain, const mmd_build_opts* o, mmd_handle* h) {
  if (validate(Ain) != MMD_OK) {
    set_error("mmd_build: bad CSR header (n < 1, nnz < n, nnz >= 2^31 or null array)");
    return MMD_EINVAL;
  }
  HCSR& A = h->A0;
  A.nrows = A.ncols = Ain->n;
  A.rowptr.assign(Ain->rowptr, Ain->rowptr + Ain->n + 1);
  A.col.assign(Ain->col, Ain->col + Ain->nnz);
  A.val.assign(Ain->val, Ain->val + Ain->nnz);
  // structural checks
  if (A.rowptr[0] != 0 || A.rowptr[A.nrows] != Ain->nnz) {
    set_error("mmd_build: rowptr[0] must be 0 and rowptr[n] = nnz");
    return MMD_EINVAL;
  }
  double amax = 0;
  for (int64_t r = 0; r < A.nrows; ++r) {
    if (A.rowptr[r + 1] < A.rowptr[r]) {
      set_error("mmd_build: rowptr not monotone");
      return MMD_EINVAL;
    }
    bool diag = false;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      const int32_t c = A.col[k];
      if (c < 0 || c >= A.nrows || (k > A.rowptr[r] && A.col[k - 1] >= c)) {
        set_error("mmd_build: column index out of range, unsorted or duplicated in row " + std::to_string(r));
        return MMD_EINVAL;
      }
      if (!std::isfinite(A.val[k])) {
        set_error("mmd_build: non-finite value in row " + std::to_string(r));
        return MMD_EINVAL;
      }
      if (c == r) {
        diag = true;
        if (!(A.val[k] > 0)) {
          set_error("mmd_build: non-positive diagonal in row " + std::to_string(r));
          return MMD_ENOTSPD;
        }
      }
      amax = std::max(amax, std::fabs(A.val[k]));
    }
    if (!diag) {
      set_error("mmd_build: missing diagonal entry in row " + std::to_string(r));
      return MMD_EINVAL;
    }
  }
  for (int64_t r = 0; r < A.nrows; ++r)
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      const int32_t c = A.col[k];
      if (c <= r) continue;
      const int32_t* b = A.col.data() + A.rowptr[c];
      const int32_t* e = A.col.data() + A.rowptr[c + 1];
      const int32_t* p = std::lower_bound(b, e, (int32_t)r);
      if (p == e || *p != r || std::fabs(A.val[p - A.col.data()] - A.val[k]) > 1e-12 * amax) {
        set_error("mmd_build: matrix is not symmetric at (" + std::to_string(r) + "," + std::to_string(c) + ")");
        return MMD_EINVAL;
      }
    }
  double ninf = 0;
  for (int64_t r = 0; r < A.nrows; ++r) {
    double s = 0;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) s += std::fabs(A.val[k]);
    ninf = std::max(ninf, s);
  }
  h->normA_inf = ninf;

  const int nt = nthreads_of(o);
  const HCSR* cur = &A;
  HCSR Mcur_id;  // identity for M^(0)
  bool have_M = false;
  h->levels.clear();
  h->levels.reserve(o->k_max);
  const char* dbg = getenv("MMD_DEBUG");
  const bool debug = dbg && dbg[0] && dbg[0] != '0';
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  while (cur->nrows > o->n_coarse && (int)h->levels.size() < o->k_max) {
    HLevel L;
    L.n_fine = cur->nrows;
    const auto t0 = now();
    partition(*cur, o->s_max, L.patch_of, L.patch_ptr, L.patch_rows);
    peel_patches(*cur, o->peel, L.patch_of, L.patch_ptr, L.patch_rows, nt);
    L.n = (int64_t)L.patch_ptr.size() - 1;
    if (L.n >= cur->nrows) break;
    bool ok = true;
    const auto t1 = now();
    local_bases(*cur, L.patch_ptr, L.patch_rows, L.patch_of, L.phi, L.uhat, L.eps, L.delta, L.used_closed, ok, nt);
    const auto t2 = now();
    if (!ok) {
      set_error("mmd_build: a patch matrix A[S,S] is not positive definite at level " +
                std::to_string(h->levels.size() + 1));
      return MMD_ENOTSPD;
    }
    // wider supports at level 1 only: the Galerkin matrices of deeper levels
    // are dense enough that two rings reach omega_max
    const int radius = h->levels.empty() ? o->loc_radius : std::min(o->loc_radius, 1);
    neighbourhoods(*cur, L.patch_of, L.patch_ptr, L.patch_rows, o->omega_max, radius, L.omega_ptr, L.omega_rows,
                   nt);
    const auto t3 = now();
    std::vector<double> psival;
    if (o->device && o->gpu_psi) {
      std::vector<double> phi_of_row(cur->nrows);
      for (int64_t x = 0; x < cur->nrows; ++x) phi_of_row[L.patch_rows[x]] = L.phi[x];
      std::string err;
      const int g = psi_solves_gpu(*cur, L.patch_of, phi_of_row, L.omega_ptr, L.omega_rows, L.n, psival, err);
      if (g != 0) {
        set_error("mmd_build: " + err + " at level " + std::to_string(h->levels.size() + 1));
        return g > 0 ? MMD_ENOTSPD : MMD_ECUDA;
      }
    } else if (!localized_psi(*cur, L.patch_of, L.phi, L.patch_rows, L.omega_ptr, L.omega_rows, L.n, psival, nt)) {
      set_error("mmd_build: a neighbourhood matrix is not positive definite at level " +
                std::to_string(h->levels.size() + 1));
      return MMD_ENOTSPD;
    }
    const auto t4 = now();
    psi_to_csr(L.n_fine, L.n, L.omega_ptr, L.omega_rows, psival, L.psi);
    HCSR PsiT, T;
    transpose(L.psi, PsiT);
    spgemm(*cur, L.psi, T, nt);
    spgemm(PsiT, T, L.A, nt);
    symmetrise(L.A);
    if (!have_M) {
      spgemm(PsiT, L.psi, L.M, nt);
    } else {
      HCSR T2;
      spgemm(h->levels.back().M, L.psi, T2, nt);
      spgemm(PsiT, T2, L.M, nt);
    }
    symmetrise(L.M);
    have_M = true;
    if (debug)
      fprintf(stderr,
              "[mmd] build level %zu: n %lld -> %lld, partition %.1f ms, bases %.1f ms, supports %.1f ms, "
              "psi %.1f ms, Galerkin %.1f ms (omega rows %zu)\n",
              h->levels.size() + 1, (long long)L.n_fine, (long long)L.n, ms(t0, t1), ms(t1, t2), ms(t2, t3),
              ms(t3, t4), ms(t4, now()), L.omega_rows.size());
    h->levels.push_back(std::move(L));
    cur = &h->levels.back().A;
  }
  (void)Mcur_id;
  return MMD_OK;
}

}  // namespace mmd
