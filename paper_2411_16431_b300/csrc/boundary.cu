// Boundary-MPS contraction of the Boltzmann-weight PEPS (paper Sec. III.B,
// Figs. 5-8), double precision.
//
// Conventions (shared with the branch step):
//  * psi_r (r = 0..R-1) stands for rows r+1..R-1; its physical index at
//    column c is the class of site (r+1, c) restricted to the spins coupled to
//    row r ("up exposure", Column::nSig); psi_{R-1} is the trivial MPS.
//  * MPO bond (c, c+1) of row r carries (lam, g): lam = left exposure of site
//    (r, c+1) (its spins coupled to (r, c) or (r+1, c)), g = class of site
//    (r+1, c+1) toward (r, c).  Diagonal couplings therefore travel on the
//    horizontal bond -- the job of the mediating tensors of Fig. 5.
//  * Sparse site diagram (Fig. 7b):  Theta[(bl, al), (u, k')] =
//      sum_{x: Lam(x)=lam, U(x)=u} w_x sum_e Ahat[(pd_x, e, g)] Ktil[(pr_x, e, pdr_x)]
//    with the projected MPS Ahat = Wa A  (bond factors to the row below
//    applied, Wa[(pd,e,g), sigma] = [pi_ul sigma = g] Bv[pd, pi_u sigma] Bdl[e, pi_ur sigma])
//    and the absorbed right tensor Ktil = Wk K (Wk[(pr,e,pdr), (lam',g')] =
//    [pi_dl lam' = e] Bh[pr, pi_l lam'] Bdr[pdr, g']).  Cost 2 chi^3 per term.
//  * Zipper (Fig. 8c): right to left from a 1x1x1 connecting tensor, SVD of
//    Theta keeping 2 chi values; then one-site variational sweeps (Fig. 8d),
//    an SVD cut to chi and more sweeps.  Singular values below 1e-12 of the
//    largest are dropped everywhere, orthonormalisations included.
//  * MPS tensors are stored [phys][bond_l][bond_r]; the approximation being
//    built (phi) is kept bond-major [bond_l][phys][bond_r].
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>

#include "handle.h"

#include "rowstep.h"

namespace sgtn {

namespace {
struct PoolKey {
  cudaStream_t st;
  size_t bytes;
  bool operator<(const PoolKey& o) const { return st != o.st ? st < o.st : bytes < o.bytes; }
};
// One cache for all streams, guarded by g_pool_mu; the stream a block is
// handed out for belongs to the calling thread.
std::recursive_mutex g_pool_mu;
std::map<PoolKey, std::vector<void*>> g_pool_free;
std::map<void*, PoolKey> g_pool_live;
size_t g_pool_cached = 0;
thread_local cudaStream_t g_pool_stream = nullptr;
constexpr size_t kPoolCap = size_t(16) << 30;   // cached bytes kept at most
size_t pool_round(size_t b) {
  if (b <= 256) return 256;
  if (b <= (size_t(1) << 20)) {
    size_t r = 256;
    while (r < b) r <<= 1;
    return r;
  }
  const size_t mb = size_t(1) << 20;
  return (b + mb - 1) / mb * mb;
}
void pool_release_all() {
  for (auto& kv : g_pool_free)
    for (void* p : kv.second) cudaFree(p);
  g_pool_free.clear();
  g_pool_cached = 0;
}
}  // namespace

void pool_set_stream(cudaStream_t st) { g_pool_stream = st; }

void* pool_alloc(size_t bytes) {
  std::lock_guard<std::recursive_mutex> lk(g_pool_mu);
  const PoolKey key{g_pool_stream, pool_round(bytes)};
  void* p = nullptr;
  auto it = g_pool_free.find(key);
  if (it != g_pool_free.end() && !it->second.empty()) {
    p = it->second.back();
    it->second.pop_back();
    g_pool_cached -= key.bytes;
  } else if (lib_malloc(&p, key.bytes) != cudaSuccess) {
    cudaGetLastError();
    pool_release_all();   // cudaFree synchronises: no cached block is still in use
    SGTN_CUDA(lib_malloc(&p, key.bytes));
  }
  g_pool_live[p] = key;
  return p;
}

void pool_free(void* p) {
  if (!p) return;
  std::lock_guard<std::recursive_mutex> lk(g_pool_mu);
  auto it = g_pool_live.find(p);
  if (it == g_pool_live.end()) {
    cudaFree(p);
    return;
  }
  const PoolKey key = it->second;
  g_pool_live.erase(it);
  if (g_pool_cached + key.bytes > kPoolCap) {
    cudaFree(p);
    return;
  }
  g_pool_free[key].push_back(p);
  g_pool_cached += key.bytes;
}

void pool_trim(cudaStream_t st) {
  std::lock_guard<std::recursive_mutex> lk(g_pool_mu);
  for (auto it = g_pool_free.begin(); it != g_pool_free.end();) {
    if (it->first.st == st) {
      for (void* p : it->second) cudaFree(p);
      g_pool_cached -= it->first.bytes * it->second.size();
      it = g_pool_free.erase(it);
    } else {
      ++it;
    }
  }
}

namespace detail {

// Linear algebra of the truncation (SVDs, orthonormalisations, canonical forms)
// always runs in FP64, also when the contractions are FP32.
struct F64Scope {
  bool saved, saved_tc;
  F64Scope() : saved(g_compute_f32), saved_tc(g_use_tc) {
    g_compute_f32 = false;
    g_use_tc = false;
  }
  ~F64Scope() {
    g_compute_f32 = saved;
    g_use_tc = saved_tc;
  }
};

// Optional per-call-site timing of the truncation linear algebra (SGTN_PROFILE
// set): each svd() call is bracketed by stream synchronisations and its wall
// time booked under the enclosing TagScope.
struct SvdProf {
  double ms = 0;
  long long calls = 0, iters = 0;
  int max_m = 0, max_n = 0;
};
// (profiling is meant for one handle at a time; the map is still guarded)
static std::map<std::string, SvdProf> g_prof;
static std::mutex g_prof_mu;
static thread_local const char* g_tag = "other";
static SvdProf& prof_entry(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof[key];
}
static bool prof_on() {
  static const bool on = std::getenv("SGTN_PROFILE") != nullptr;
  return on;
}
struct TagScope {
  const char* saved;
  explicit TagScope(const char* t) : saved(g_tag) { g_tag = t; }
  ~TagScope() { g_tag = saved; }
};

double* dmalloc(long long n) { return static_cast<double*>(pool_alloc(size_t(n > 0 ? n : 1) * sizeof(double))); }
void dfree(double*& p) {
  pool_free(p);
  p = nullptr;
}

double norm_host(sgtn_inst* h, const double* x, long long n, bool allow_zero);
SvdOut svd_dense(sgtn_inst* h, const double* Th, int m, int n, int cap);
double* left_factor(sgtn_inst* h, const SvdOut& o, int m);
SvdOut svd_subspace(sgtn_inst* h, const double* Th, int m, int n, int cap);
using MatFn = std::function<void(const double* Q, int s, double* Y)>;
SvdOut svd_subspace_op(sgtn_inst* h, int m, int n, int cap, const MatFn& mul, const MatFn& tmul);

// Truncated SVD of a dense row-major m x n matrix: exact one-sided Jacobi on
// the shorter side when it is short, otherwise subspace iteration with a
// Rayleigh-Ritz step (converged to the same top singular subspace).
SvdOut svd_impl(sgtn_inst* h, const double* Th, int m, int n, int cap) {
  F64Scope f64;
  int p = std::min(m, n);
  if (p <= h->dense_svd_max || cap >= p) return svd_dense(h, Th, m, n, cap);
  return svd_subspace(h, Th, m, n, cap);
}

template <class F>
auto profiled(sgtn_inst* h, const char* sub, int m, int n, F&& f) -> decltype(f()) {
  if (!prof_on()) return f();
  h->sync();
  auto t0 = std::chrono::steady_clock::now();
  auto o = f();
  h->sync();
  SvdProf& e = prof_entry(std::string(g_tag) + sub);
  e.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  e.calls += 1;
  e.max_m = std::max(e.max_m, m);
  e.max_n = std::max(e.max_n, n);
  return o;
}

SvdOut svd(sgtn_inst* h, const double* Th, int m, int n, int cap) {
  return profiled(h, "", m, n, [&] { return svd_impl(h, Th, m, n, cap); });
}

SvdOut svd_jacobi(sgtn_inst* h, const double* Th, int m, int n, int cap);
bool cqr_orth(sgtn_inst* h, const double* M, int len, int k, double* Q, bool first_f32);
bool orth_qr(sgtn_inst* h, const double* M, int m, int n, bool rows, double* Q);
bool svd_tall_cqr(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o);
bool svd_tall_cqr3(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o);
bool svd_tall_rrcqr(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o);

// Exact truncated SVD: for a matrix with a short side of at most 320 (and a
// long side of at least 256, or a short side of at least 64), CholeskyQR2 or
// shifted CholeskyQR3 then a one-sided Jacobi SVD of the rows of the small
// triangular factor (rank-revealing CholeskyQR for dependent vectors,
// up to 160 of them); a truncation well below the short side of dependent
// vectors goes to subspace iteration; otherwise one-sided Jacobi on the
// shorter side.
SvdOut svd_dense(sgtn_inst* h, const double* Th, int m, int n, int cap) {
  SvdOut o;
  int p = std::min(m, n), q = std::max(m, n);
  // CholeskyQR first also for squarish matrices of 64 or more vectors: the
  // one-sided Jacobi then rotates the rows of the triangular factor, which
  // converges in about a third of the sweeps that the vectors of a matrix
  // with graded singular values take
  if (p <= 320 && (q >= 256 || p >= 64)) {
    if (prof_on()) prof_entry(std::string(g_tag) + "/cqr_tries").calls++;
    if (m >= n) {
      if (svd_tall_cqr(h, Th, m, n, cap, o)) return o;
    } else {
      // M (m x n, short-fat): factor M^T = U S V^T, then M = V S U^T
      double* Mt = h->ws.get<double>("svd_Mt", size_t(m) * n);
      int dims[2] = {m, n}, perm[2] = {1, 0};
      permute_nd(Th, 2, dims, perm, Mt, h->st);
      SvdOut t;
      if (svd_tall_cqr(h, Mt, n, m, cap, t)) {
        o.k = t.k;
        o.sig = t.sig;
        o.dsig = t.dsig;
        t.dsig = nullptr;
        // US(M) = (Vt_t)^T S : m x k ; Vt(M) = (US_t / S)^T : k x n
        o.US = dmalloc((long long)m * o.k);
        gather_vecs(t.Vt, m, 1, m, h->iota, o.dsig, o.k, o.US, o.k, 1, h->st);
        o.Vt = dmalloc((long long)o.k * n);
        gather_vecs(t.US, n, t.k, 1, h->iota, o.dsig + o.k, o.k, o.Vt, 1, n, h->st);
        t.release();
        return o;
      }
    }
    // numerically dependent vectors, too many for the pivoted Cholesky: a
    // truncation to well below the short side takes the leading subspace by
    // subspace iteration (a few products with Theta) instead of rotating all
    // p long vectors to convergence
    if (cap + 32 < p) {
      if (prof_on()) prof_entry(std::string(g_tag) + "/dependent_subspace").calls++;
      return svd_subspace(h, Th, m, n, cap);
    }
  }
  return svd_jacobi(h, Th, m, n, cap);
}

// M (m x n, m >= n, row-major) = Q R by CholeskyQR2 (well-conditioned M) or
// shifted CholeskyQR3, then R = U S V^T by one-sided Jacobi.  Returns false
// (nothing allocated) if a pivot fails (numerically dependent columns).
bool svd_tall_cqr3(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o) {
  cudaStream_t st = h->st;
  double* G = h->ws.get<double>("cq_G", size_t(n) * n);
  double* G0 = h->ws.get<double>("cq_G0", size_t(n) * n);
  double* R = h->ws.get<double>("cq_R", size_t(n) * n);
  double* Ri = h->ws.get<double>("cq_Ri", size_t(n) * n);
  double* Racc = h->ws.get<double>("cq_Racc", size_t(n) * n);
  double* Rtmp = h->ws.get<double>("cq_Rtmp", size_t(n) * n);
  double* Qa = h->ws.get<double>("cq_Qa", size_t(m) * n);
  double* Qb = h->ws.get<double>("cq_Qb", size_t(m) * n);
  double* dmr = h->ws.get<double>("cq_minratio", 1);
  int* status = h->ws.get<int>("cq_status", 4);
  SGTN_CUDA(cudaMemsetAsync(status, 0, 3 * sizeof(int), st));
  // one pass: G = cur^T cur, R = chol(G + shift I), out = cur R^{-1}, Racc = R Racc
  auto pass = [&](const double* cur, double* out, double shift, int* stat, bool first, const double* Gin) {
    if (!Gin) gram_upper(cur, n, G, n, m, st);
    cholesky_inv(Gin ? Gin : G, n, shift, R, Ri, stat, st);
    gemm(cur, false, n, Ri, false, n, out, n, m, n, n, 1.0, 0, st, 2);
    if (first) {
      copy(Racc, R, (long long)n * n, st);
    } else {
      gemm(R, false, n, Racc, false, n, Rtmp, n, n, n, n, 1.0, 0, st, 2);
      copy(Racc, Rtmp, (long long)n * n, st);
    }
  };
  gram_upper(M, n, G0, n, m, st);
  // CholeskyQR2 when the unshifted factor lost at most 10 of the 16 digits of
  // any column (cond(M) below about 1e5): its orthogonality after two passes
  // is at rounding level
  cholesky_inv(G0, n, 0.0, R, Ri, status, st, false, dmr);
  std::vector<double> hdiag(n);
  double mr = 0;
  int hs0 = 0;
  SGTN_CUDA(cudaMemcpy2DAsync(hdiag.data(), sizeof(double), G0, size_t(n + 1) * sizeof(double), sizeof(double), n,
                              cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(&mr, dmr, sizeof(double), cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(&hs0, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  h->sync();
  double tr = 0;
  for (int i = 0; i < n; ++i) tr += hdiag[i];
  if (!(tr > 0) || !std::isfinite(tr)) return false;
  const double* cur = nullptr;
  if (hs0 == 0 && mr > 1e-10) {
    gemm(M, false, n, Ri, false, n, Qa, n, m, n, n, 1.0, 0, st, 2);              // Q1 = M R1^{-1}
    copy(Racc, R, (long long)n * n, st);
    pass(Qa, Qb, 0.0, status + 1, false, nullptr);
    cur = Qb;
  } else {
    // shifted CholeskyQR3: first shift 11 (m n + n (n+1)) eps ||M||_2^2, with
    // ||M||_2^2 <= trace(M^T M)
    const double shift = 11.0 * (double(m) * n + double(n) * (n + 1)) * 2.220446049250313e-16 * tr;
    SGTN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    pass(M, Qa, shift, status, true, G0);
    pass(Qa, Qb, 0.0, status + 1, false, nullptr);
    pass(Qb, Qa, 0.0, status + 2, false, nullptr);
    cur = Qa;
  }
  int hs[3] = {0, 0, 0};
  SGTN_CUDA(cudaMemcpyAsync(hs, status, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  h->sync();
  if (hs[0] || hs[1] || hs[2]) return false;
  // SVD of the n x n factor: Racc V = W, sigma = |W_j|
  SvdOut r = svd_jacobi(h, Racc, n, n, cap);
  // M = Q Racc = (Q U_R) S V^T :  US = Q (U_R S) = Q r.US ; Vt = r.Vt
  o.k = r.k;
  o.sig = r.sig;
  o.dsig = r.dsig;
  r.dsig = nullptr;
  o.Vt = r.Vt;
  r.Vt = nullptr;
  o.US = dmalloc((long long)m * o.k);
  gemm(cur, false, n, r.US, false, o.k, o.US, o.k, m, o.k, n, 1.0, 0, st);
  r.release();
  return true;
}

// Tall-skinny SVD: shifted CholeskyQR3 (the exact path), or, when its
// Cholesky factor fails (numerically dependent columns), rank-revealing
// CholeskyQR; false if both fail.
bool svd_tall_cqr(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o) {
  if (svd_tall_cqr3(h, M, m, n, cap, o)) return true;
  if (n > 160) return false;   // the pivoted Cholesky is staged in one CTA's shared memory
  if (prof_on()) prof_entry(std::string(g_tag) + "/rrcqr").calls++;
  return svd_tall_rrcqr(h, M, m, n, cap, o);
}

// M (m x n, m >= n, row-major) = Q B with Q (m x r) orthonormal and r the
// numerical rank, then B = U S V^T by one-sided Jacobi, so M = (Q U) S V^T.
// Q is built in at most three rounds of rank-revealing CholeskyQR: pivoted
// Cholesky of the Gram matrix of the current residual (stopped where the
// remaining pivots fall below 1e-14 of the largest, i.e. residual columns
// below 1e-7 of the largest norm), Q1 = M[:, piv] R^{-1} made orthogonal to the
// earlier columns and orthonormalised by CholeskyQR2; B = Q^T M and the
// residual M - Q B decide whether another round is needed (its Frobenius norm
// above 1e-14 of ||M||_F).  Returns false (nothing allocated) if a round fails.
// Used where shifted CholeskyQR3 fails; it is slightly less accurate there.
bool svd_tall_rrcqr(sgtn_inst* h, const double* M, int m, int n, int cap, SvdOut& o) {
  cudaStream_t st = h->st;
  double* G = h->ws.get<double>("cq_G", size_t(n) * n);
  double* R = h->ws.get<double>("cq_R", size_t(n) * n);
  double* Ri = h->ws.get<double>("cq_Ri", size_t(n) * n);
  double* Qt = h->ws.get<double>("cq_Qt", size_t(m) * n);     // Q total, leading dimension n
  double* Mp = h->ws.get<double>("cq_Mp", size_t(m) * n);
  double* Q1 = h->ws.get<double>("cq_Q1", size_t(m) * n);
  double* Q2 = h->ws.get<double>("cq_Q2", size_t(m) * n);
  double* E = h->ws.get<double>("cq_E", size_t(m) * n);
  double* B = h->ws.get<double>("cq_B", size_t(n) * n);
  double* C = h->ws.get<double>("cq_C", size_t(n) * n);
  double* ones = h->ws.get<double>("cq_ones", n);
  int32_t* perm = h->ws.get<int32_t>("cq_perm", n);
  int* rank = h->ws.get<int>("cq_rank", 1);
  fill(ones, n, 1.0, st);
  const double normM = norm_host(h, M, (long long)m * n, true);
  if (!(normM > 0.0)) return false;
  double floor_abs = 0.0;
  const double* cur = M;   // residual whose range is being added
  int rt = 0;
  for (int round = 0; round < 3 && rt < n; ++round) {
    gemm(cur, true, n, cur, false, n, G, n, n, n, m, 1.0, 0, st);                       // G = cur^T cur
    if (round == 0) {
      // absolute floor for later rounds: pivots of (1e-13 max column norm)^2
      std::vector<double> d(n);
      SGTN_CUDA(cudaMemcpy2DAsync(d.data(), sizeof(double), G, size_t(n + 1) * sizeof(double), sizeof(double), n,
                                  cudaMemcpyDeviceToHost, st));
      h->sync();
      double dm = 0;
      for (double v : d) dm = std::max(dm, v);
      floor_abs = 1e-26 * dm;
    }
    pchol_inv(G, n, 1e-14, floor_abs, R, Ri, perm, rank, st);
    int r = 0;
    SGTN_CUDA(cudaMemcpyAsync(&r, rank, sizeof(int), cudaMemcpyDeviceToHost, st));
    h->sync();
    r = std::min(r, n - rt);
    if (r <= 0) break;
    // Q1 = cur[:, perm] R^{-1}
    gather_vecs(cur, m, n, 1, perm, ones, r, Mp, r, 1, st);
    gemm(Mp, false, r, Ri, false, n, Q1, r, m, r, r, 1.0, 0, st, 2);
    if (rt > 0) {
      // Q1 -= Qt (Qt^T Q1), twice (classical Gram-Schmidt with reorthogonalisation)
      for (int pass = 0; pass < 2; ++pass) {
        gemm(Qt, true, n, Q1, false, r, C, r, rt, r, m, 1.0, 0, st);
        gemm(Qt, false, n, C, false, r, Q1, r, m, r, rt, -1.0, 1, st);
      }
    }
    if (!cqr_orth(h, Q1, m, r, Q2, false)) return false;
    gather_vecs(Q2, m, r, 1, h->iota, ones, r, Qt + rt, n, 1, st);                     // append columns
    rt += r;
    if (rt >= n) break;
    // B = Qt^T M ; E = M - Qt B
    gemm(Qt, true, n, M, false, n, B, n, rt, n, m, 1.0, 0, st);
    gemm(Qt, false, n, B, false, n, E, n, m, n, rt, -1.0, 0, st);
    add_cols(E, M, m, n, n, st);
    const double ne = norm_host(h, E, (long long)m * n, true);
    if (!(ne > 1e-14 * normM)) break;
    cur = E;
  }
  if (rt <= 0) return false;
  gemm(Qt, true, n, M, false, n, B, n, rt, n, m, 1.0, 0, st);                          // B = Qt^T M (rt x n)
  SvdOut r = svd_jacobi(h, B, rt, n, cap);
  // M = Qt B = (Qt U_B) S V^T :  US = Qt r.US ; Vt = r.Vt
  o.k = r.k;
  o.sig = r.sig;
  o.dsig = r.dsig;
  r.dsig = nullptr;
  o.Vt = r.Vt;
  r.Vt = nullptr;
  o.US = dmalloc((long long)m * o.k);
  gemm(Qt, false, n, r.US, false, o.k, o.US, o.k, m, o.k, rt, 1.0, 0, st);
  r.release();
  return true;
}

// Exact truncated SVD by one-sided Jacobi on the shorter side.
SvdOut svd_jacobi(sgtn_inst* h, const double* Th, int m, int n, int cap) {
  cudaStream_t st = h->st;
  SvdOut o;
  double* T2 = h->ws.get<double>("svd_T2", size_t(m) * n);
  copy(T2, Th, (long long)m * n, st);
  int* status = h->ws.get<int>("svd_status", 1);
  int p = std::min(m, n);
  double* dsigall = h->ws.get<double>("svd_sig", p);
  double* V = nullptr;
  if (prof_on()) h->sync();
  auto t0 = std::chrono::steady_clock::now();
  if (m <= n) {
    // the rows are the vectors; V (m x m) accumulates the rotations, so the
    // left factor comes out exactly orthogonal (U = V), also for directions
    // with tiny singular values
    V = h->ws.get<double>("svd_V", size_t(m) * m);
    jacobi(T2, n, m, 1, n, V, 60, status, st);
    vec_norms(T2, n, m, 1, n, dsigall, st);
  } else {
    V = h->ws.get<double>("svd_V", size_t(n) * n);
    jacobi(T2, m, n, n, 1, V, 60, status, st);
    vec_norms(T2, m, n, n, 1, dsigall, st);
  }
  h->check();
  std::vector<double> s(p);
  int hs = 0;
  SGTN_CUDA(cudaMemcpyAsync(s.data(), dsigall, p * sizeof(double), cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  h->sync();
  if (hs < 0) throw SgtnError(-4, "Jacobi SVD did not converge");
  {
    // per sweep: the squared norms (2 flop per element), and per pair the
    // product (2 flop per element), the rotation of both vectors (6) and of
    // their columns of V (6 per element of V)
    const double vl = std::max(m, n), np = p;
    ktimer_add_flops("jacobi_f64", double(hs) * (2.0 * np * vl + np * (np - 1) / 2 * (8.0 * vl + 6.0 * np)));
  }
  if (prof_on()) {
    SvdProf& e = prof_entry(std::string(g_tag) + (std::max(m, n) > 128 ? "/jacobi_long" : "/jacobi"));
    e.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    e.calls++;
    e.iters += hs;
    e.max_m = std::max(e.max_m, p);
    e.max_n = std::max(e.max_n, std::max(m, n));
  }
  std::vector<int> idx(p);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s[a] > s[b]; });
  double smax = p ? s[idx[0]] : 0.0;
  if (std::getenv("SGTN_TRACE"))
    fprintf(stderr, "[sgtn] svd_jacobi m=%d n=%d cap=%d smax=%.3e smin=%.3e sweeps=%d ms=%.3f\n", m, n, cap, smax,
            p ? s[idx[p - 1]] : 0.0, hs,
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  if (!(smax > 0.0) || !std::isfinite(smax)) throw SgtnError(-4, "zero or non-finite tensor in truncation");
  int cnt = 0;
  for (int i = 0; i < p; ++i)
    if (s[idx[i]] > RANK_TOL * smax) ++cnt;
  int k = std::min(cap, cnt);
  o.k = k;
  std::vector<double> sv(2 * k);
  std::vector<int32_t> perm(k);
  for (int i = 0; i < k; ++i) {
    perm[i] = idx[i];
    sv[i] = s[idx[i]];
    sv[k + i] = 1.0 / s[idx[i]];
    o.sig.push_back(s[idx[i]]);
  }
  int32_t* dperm = h->ws.get<int32_t>("svd_perm", k);
  o.dsig = dmalloc(2 * k);
  SGTN_CUDA(cudaMemcpyAsync(dperm, perm.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SGTN_CUDA(cudaMemcpyAsync(o.dsig, sv.data(), 2 * k * sizeof(double), cudaMemcpyHostToDevice, st));
  o.US = dmalloc((long long)m * k);
  o.Vt = dmalloc((long long)k * n);
  if (m <= n) {
    gather_vecs(T2, n, 1, n, dperm, o.dsig + k, k, o.Vt, 1, n, st);        // rows / sigma
    gather_vecs(V, m, 1, m, dperm, o.dsig, k, o.US, k, 1, st);             // U S = V diag(sigma)
  } else {
    double* ones = h->ws.get<double>("svd_ones", k);
    fill(ones, k, 1.0, st);
    gather_vecs(V, n, 1, n, dperm, ones, k, o.Vt, 1, n, st);
    gather_vecs(T2, m, n, 1, dperm, ones, k, o.US, k, 1, st);
  }
  h->check();
  // the host waits on the next transfer anyway; keep perm alive until then
  h->sync();
  return o;
}

// Top-k right singular subspace of Theta (m x n) by block subspace iteration:
// Q <- orth(Theta^T orth(Theta Q)) with a block of s = min(p, k + 32) vectors
// from a fixed pseudo-random start, until the leading Ritz vectors (weighted by
// their singular values) settle; the Rayleigh-Ritz step (SVD of Theta Q, s
// columns, exact) gives the singular values and Q W the vectors.
SvdOut svd_subspace(sgtn_inst* h, const double* Th, int m, int n, int cap) {
  MatFn mul = [=](const double* Q, int s, double* Y) { gemm(Th, false, n, Q, false, s, Y, s, m, s, n, 1.0, 0, h->st); };
  MatFn tmul = [=](const double* Y, int s, double* Z) { gemm(Th, true, n, Y, false, s, Z, s, n, s, m, 1.0, 0, h->st); };
  return svd_subspace_op(h, m, n, cap, mul, tmul);
}

// Orthonormal basis of the columns of M (len x k, row-major) into Q by
// CholeskyQR passes (Gram matrix, Cholesky factor R, multiplication by R^{-1}),
// repeated until the Gram matrix of a pass's input lies within 0.1 of the
// identity: that pass leaves an orthogonality error of a few ulps
// (CholeskyQR2; a shifted first factor when the unshifted one fails, as in
// shifted CholeskyQR3).  first_f32: the first factor in FP32 arithmetic (the
// FP64 passes after it remove its rounding).  Returns false if a pivot of a
// later pass fails (numerically dependent columns); Q is then unspecified.
// Q must not alias M.
bool cqr_orth(sgtn_inst* h, const double* M, int len, int k, double* Q, bool first_f32) {
  F64Scope f64;
  cudaStream_t st = h->st;
  if (k < 1 || len < k) return false;
  double* G = h->ws.get<double>("cqo_G", size_t(k) * k);
  double* R = h->ws.get<double>("cqo_R", size_t(k) * k);
  double* Ri = h->ws.get<double>("cqo_Ri", size_t(k) * k);
  double* T = h->ws.get<double>("cqo_T", size_t(len) * k);
  double* T2 = h->ws.get<double>("cqo_T2", size_t(len) * k);
  int* status = h->ws.get<int>("cqo_status", 1);
  // deviation of the Gram matrix from the identity and its trace, computed on
  // the device and read with the Cholesky status (one transfer of 16 bytes)
  double* dstat = h->ws.get<double>("cqo_stat", 2);
  double hstat[2] = {0.0, 0.0};
  auto chol = [&](double shift, bool f32) {
    cholesky_inv(G, k, shift, R, Ri, status, st, f32);
    int hs = 0;
    SGTN_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGTN_CUDA(cudaMemcpyAsync(hstat, dstat, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    h->sync();
    return hs == 0;
  };
  const double* cur = M;
  for (int pass = 0; pass < 4; ++pass) {
    // G = cur^T cur (upper).  A first factor taken in FP32 only preconditions
    // (the FP64 passes after it restore orthogonality, and cur R^{-1} keeps
    // the span exactly), so its Gram matrix is formed in FP32 too: the
    // product of the tall operand is the costliest step of the pass
    const bool g32 = pass == 0 && first_f32;
    if (g32) g_compute_f32 = true;
    gram_upper(cur, k, G, k, len, st);
    g_compute_f32 = false;
    gram_stats(G, k, dstat, st);
    bool last = pass == 3;
    if (pass == 0) {
      bool ok = chol(0.0, first_f32);
      if (!ok && first_f32) {
        gram_upper(cur, k, G, k, len, st);                             // FP64 Gram for the FP64 factor
        gram_stats(G, k, dstat, st);
        ok = chol(0.0, false);
      }
      if (!ok) {
        const double tr = hstat[1];
        if (!(tr > 0) || !std::isfinite(tr)) return false;
        double shift = 11.0 * (double(len) * k + double(k) * (k + 1)) * 2.220446049250313e-16 * tr;
        if (!chol(shift, false)) return false;
      }
    } else {
      if (!chol(0.0, false)) return false;
      const double dev = hstat[0];
      if (!std::isfinite(dev)) return false;
      last = last || dev < 0.1;
    }
    double* out = last ? Q : (cur == T ? T2 : T);
    gemm(cur, false, k, Ri, false, k, out, k, len, k, k, 1.0, 0, st, 2);   // out = cur R^{-1}
    cur = out;
    if (last) break;
  }
  h->check();
  return true;
}

// Orthonormal basis of the span of M by CholeskyQR, for the orthonormalisations
// of the variational sweeps, where only the span matters (the next one-site
// update projects the target onto it again) and no truncation is asked for.
// rows = false: M is m x n (m >= n), Q (m x n) gets orthonormal columns with
// the column span of M; rows = true: M is m x n (m <= n), Q (m x n) gets
// orthonormal rows with the row space of M.  Taken only when the truncated SVD
// would keep every direction: the unshifted FP64 Cholesky factor R of the
// Gram matrix succeeds with every pivot above 1e-10 of its diagonal entry (a
// scale-invariant condition under which two passes reach rounding-level
// orthogonality, also for vectors of very different norms) and
// ||M||_F ||R^{-1}||_F -- an upper bound on sigma_max / sigma_min, since
// sigma_max <= ||M||_F and 1 / sigma_min = ||R^{-1}||_2 <= ||R^{-1}||_F --
// stays below 1 / RANK_TOL, so the rank rule would drop nothing.  The first
// pass leaves vectors Q1 whose Gram matrix is I + E with |E| about
// cond^2 x 1e-16; instead of a second Cholesky pass, one step of the Newton
// iteration for the polar factor, Q = Q1 (3 I - Q1^T Q1) / 2, leaves an
// orthogonality error of O(|E|^2), accepted when max |E| <= 1e-6 (so at most
// about 1e-12; well-conditioned vectors reach rounding level).  Returns false
// otherwise (the caller then takes the SVD); Q is then unspecified.
bool orth_qr(sgtn_inst* h, const double* M, int m, int n, bool rows, double* Q) {
  F64Scope f64;
  cudaStream_t st = h->st;
  const int k = rows ? m : n, len = rows ? n : m;   // k vectors of length len
  if (k < 1 || len < k || k > h->dense_svd_max) return false;
  double* G = h->ws.get<double>("oq_G", size_t(k) * k);
  double* R = h->ws.get<double>("oq_R", size_t(k) * k);
  double* Ri = h->ws.get<double>("oq_Ri", size_t(k) * k);
  double* T = h->ws.get<double>("oq_T", size_t(len) * k);
  double* dv = h->ws.get<double>("oq_vals", 4);   // minratio, max |G - I|, trace, ||R^{-1}||_F
  int* status = h->ws.get<int>("oq_status", 2);
  // upper triangle of the Gram matrix of the vectors
  auto gram = [&](const double* X) {
    if (rows) gemm(X, false, len, X, true, len, G, k, k, k, len, 1.0, 0, st, 1);
    else gram_upper(X, k, G, k, len, st);
  };
  // out = X R^{-1} (columns) or R^{-T} X (rows)
  auto apply = [&](const double* X, double* out) {
    if (rows) gemm(Ri, true, k, X, false, len, out, len, k, len, k, 1.0, 0, st);
    else gemm(X, false, k, Ri, false, k, out, k, len, k, k, 1.0, 0, st, 2);
  };
  gram(M);
  gram_stats(G, k, dv + 1, st);
  cholesky_inv(G, k, 0.0, R, Ri, status, st, false, dv);
  fro_norm(Ri, (long long)k * k, dv + 3, st);
  double hv[4];
  int hs = 0;
  SGTN_CUDA(cudaMemcpyAsync(hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  h->sync();
  // ||M||_F^2 = trace(G)
  const double bound = std::sqrt(hv[2]) * hv[3];
  if (hs != 0 || !(hv[0] > 1e-10) || !(bound < 1.0 / RANK_TOL)) return false;
  apply(M, T);
  gram(T);
  gram_stats(G, k, dv + 1, st);
  polar_factor(G, k, R, st);
  if (rows) gemm(R, false, k, T, false, len, Q, len, k, len, k, 1.0, 0, st);   // Q = S Q1
  else gemm(T, false, k, R, false, k, Q, k, len, k, k, 1.0, 0, st);            // Q = Q1 S
  double dev = 0.0;
  SGTN_CUDA(cudaMemcpyAsync(&dev, dv + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  h->sync();
  return dev <= 1e-6;
}

// Same, with Theta given only through Y = Theta Q and Z = Theta^T Y.  Each
// iteration orthonormalises both products by CholeskyQR (Y before it is
// multiplied back, so that no condition number is squared); every second
// iteration a Rayleigh-Ritz step (exact SVD of Theta Q) gives the Ritz
// vectors, and the iteration stops when the leading min(cap, k) of them,
// weighted by sigma_j / sigma_1, moved by less than 1e-13 sqrt(k) (Frobenius)
// since the previous check.
SvdOut svd_subspace_op(sgtn_inst* h, int m, int n, int cap, const MatFn& mul, const MatFn& tmul) {
  F64Scope f64;
  cudaStream_t st = h->st;
  const int p = std::min(m, n);
  const int s = std::min(p, cap + 32);
  double* Q = h->ws.get<double>("ss_Q", size_t(n) * s);
  double* Qn = h->ws.get<double>("ss_Qn", size_t(n) * s);
  double* Y = h->ws.get<double>("ss_Y", size_t(m) * s);
  double* Yq = h->ws.get<double>("ss_Yq", size_t(m) * s);
  double* Z = h->ws.get<double>("ss_Z", size_t(n) * s);
  double* G = h->ws.get<double>("ss_G", size_t(s) * s);
  double* Vp = h->ws.get<double>("ss_Vp", size_t(n) * s);
  double* ones = h->ws.get<double>("ss_ones", s);
  double* wdev = h->ws.get<double>("ss_w", s);
  fill(ones, s, 1.0, st);
  // orthonormal basis of the columns of A (len x kk) into out; dependent
  // columns (a failed pivot) go through the rank-trimmed SVD basis instead
  auto orth = [&](double* A, int len, int& kk, double* out) {
    if (cqr_orth(h, A, len, kk, out, true)) return;
    SvdOut o = svd_dense(h, A, len, kk, kk);
    gather_vecs(o.US, len, o.k, 1, h->iota, o.dsig + o.k, o.k, out, o.k, 1, st);
    kk = o.k;
    o.release();
  };
  int k = s;
  pseudo_random(Z, (long long)n * s, 12345, st);
  orth(Z, n, k, Q);
  const int maxit = 60;
  int kc_prev = -1;
  for (int it = 0;; ++it) {
    mul(Q, k, Y);                                                                 // Y = Theta Q
    const bool last = it + 1 >= maxit;
    if (it % 2 == 1 || last) {
      // Rayleigh-Ritz: Theta Q = U S W^T; Ritz vectors Q W, Ritz values S
      SvdOut ob = svd_dense(h, Y, m, k, k);
      const int kb = ob.k, kc = std::min(cap, kb);
      gemm(Q, false, k, ob.Vt, true, k, Qn, kb, n, kb, k, 1.0, 0, st);           // Qn = Q W  (n x kb)
      double ch = INFINITY;
      if (kc == kc_prev) {
        // || Vp - Qn_c (Qn_c^T Vp) ||  with Qn_c the leading kc Ritz vectors and
        // the columns of Vp weighted by sigma_j / sigma_1: the change of the
        // rank-kc approximation relative to its norm (a direction whose
        // singular value sits at rounding level cannot settle, nor matters)
        double* Rr = h->ws.get<double>("ss_R", size_t(n) * kc);
        gemm(Qn, true, kb, Vp, false, kc, G, kc, kc, kc, n, 1.0, 0, st);
        gemm(Qn, false, kb, G, false, kc, Rr, kc, n, kc, kc, -1.0, 0, st);
        add_cols(Rr, Vp, n, kc, kc, st);
        ch = norm_host(h, Rr, (long long)n * kc, true);
      }
      const bool conv = ch < 1e-13 * std::sqrt(double(kc));
      if (conv || last) {
        // no gap at the cut: the truncation is ambiguous; keep the last
        // Rayleigh-Ritz result and count the cut
        if (!conv) ++h->unconverged_cuts;
        if (prof_on()) {
          SvdProf& e = prof_entry(std::string(g_tag) + "/subspace");
          e.iters += it + 1;
          e.calls++;
          if (std::getenv("SGTN_TRACE"))
            fprintf(stderr, "[sgtn] subspace m=%d n=%d cap=%d it=%d ch=%.2e s1=%.3e s_cap=%.3e s_cap+1=%.3e s_last=%.3e\n",
                    m, n, cap, it + 1, ch, ob.sig[0], ob.sig[kc - 1], kc < kb ? ob.sig[kc] : 0.0, ob.sig[kb - 1]);
        }
        SvdOut o;
        o.k = kc;
        o.sig.assign(ob.sig.begin(), ob.sig.begin() + kc);
        std::vector<double> sv(2 * kc);
        for (int i = 0; i < kc; ++i) sv[i] = o.sig[i], sv[kc + i] = 1.0 / o.sig[i];
        o.dsig = dmalloc(2 * kc);
        SGTN_CUDA(cudaMemcpyAsync(o.dsig, sv.data(), 2 * kc * sizeof(double), cudaMemcpyHostToDevice, st));
        o.US = dmalloc((long long)m * kc);
        gather_vecs(ob.US, m, kb, 1, h->iota, ones, kc, o.US, kc, 1, st);
        o.Vt = dmalloc((long long)kc * n);
        gather_vecs(Qn, n, kb, 1, h->iota, ones, kc, o.Vt, 1, n, st);
        ob.release();
        h->sync();   // sv stays alive until the copy is done
        return o;
      }
      {
        // Vp = leading kc Ritz vectors, column j scaled by sigma_j / sigma_1
        std::vector<double> w(kc);
        for (int j = 0; j < kc; ++j) w[j] = ob.sig[j] / ob.sig[0];
        SGTN_CUDA(cudaMemcpyAsync(wdev, w.data(), kc * sizeof(double), cudaMemcpyHostToDevice, st));
        gather_vecs(Qn, n, kb, 1, h->iota, wdev, kc, Vp, kc, 1, st);
        h->sync();
      }
      kc_prev = kc;
      // continue from the Ritz basis: Q = Q W, Theta Q = U S
      std::swap(Q, Qn);
      k = kb;
      copy(Y, ob.US, (long long)m * k, st);
      ob.release();
    }
    int ky = k;
    orth(Y, m, ky, Yq);
    tmul(Yq, ky, Z);                                                              // Z = Theta^T Yq
    k = ky;
    orth(Z, n, k, Q);
  }
}

void SvdOut::release() {
  dfree(US);
  dfree(Vt);
  dfree(dsig);
}

// Q = US / sigma (m x k)
double* left_factor(sgtn_inst* h, const SvdOut& o, int m) {
  double* Q = dmalloc((long long)m * o.k);
  gather_vecs(o.US, m, o.k, 1, h->iota, o.dsig + o.k, o.k, Q, o.k, 1, h->st);
  return Q;
}
// R = sigma Vt (k x n)
double* right_factor(sgtn_inst* h, const SvdOut& o, int n) {
  double* Rm = dmalloc((long long)o.k * n);
  gather_vecs(o.Vt, n, 1, n, h->iota, o.dsig, o.k, Rm, 1, n, h->st);
  return Rm;
}

// Frobenius norm of x read back to the host, as it is (0, inf or NaN included).
double norm_value(sgtn_inst* h, const double* x, long long n) {
  double* d = h->ws.get<double>("norm_out", 1);
  fro_norm(x, n, d, h->st);
  double v = 0;
  SGTN_CUDA(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  return v;
}

// Change of an adaptive weight exponent from the norm v of the result it
// produced: 0 while v lies within 2^+-100 (FP32 reaches 2^-126 in normal
// numbers; nothing is recomputed for results that are merely small), else the
// power of two that brings it near 1 (+100 for a result that underflowed to
// zero, -100 for one that overflowed).
int exp_step(double v) {
  if (!std::isfinite(v)) return -100;
  if (!(v > 0.0)) return 100;
  const int ex = std::ilogb(v);
  return (ex >= -100 && ex <= 100) ? 0 : -ex;
}

double norm_host(sgtn_inst* h, const double* x, long long n, bool allow_zero) {
  double* d = h->ws.get<double>("norm_out", 1);
  fro_norm(x, n, d, h->st);
  double v = 0;
  SGTN_CUDA(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  if (!std::isfinite(v) || (!allow_zero && !(v > 0.0))) throw SgtnError(-4, "zero or non-finite norm");
  return v;
}
// Rescale x by the power of two nearest its norm (exact: changes no digit of
// any later result, only keeps magnitudes inside the floating-point range).
void rescale_pow2(sgtn_inst* h, double* x, long long n, double& lognorm) {
  double v = norm_host(h, x, n, false);
  int e = (int)std::lround(std::log2(v));
  if (e == 0) return;
  lognorm += e * 0.69314718055994530942;
  scale_pow2(x, n, e, h->st);
}

void normalise(sgtn_inst* h, double* x, long long n, double& lognorm) {
  double v = norm_host(h, x, n, false);
  lognorm += std::log(v);
  scale_by_inv(x, n, h->ws.get<double>("norm_out", 1), h->st);
}

// Ktil = Wk * K   with K [nBR][chr][kp]
double* absorb(RowCtx& X, int c, const double* K, int kp, const char* name) {
  const Column& K_ = X.col(c);
  double* Kt = X.h->ws.get<double>(name, size_t(K_.nK()) * X.chr(c) * kp);
  gemm(K_.Wk, false, K_.nBR(), K, false, (long long)X.chr(c) * kp, Kt, (long long)X.chr(c) * kp, K_.nK(),
       X.chr(c) * kp, K_.nBR(), 1.0, 0, X.h->st);
  return Kt;
}

constexpr double kLn2 = 0.69314718055994530942;

// Exponent s of column c's weights in the current arithmetic: the FP32, TF32
// and BF16 contractions multiply by w 2^s (exact in FP64) so that products
// that would fall out of FP32's range stay in it; 0 in FP64 or without hints.
int weight_exp(const RowCtx& X, int c) { return (g_compute_f32 && X.sexp) ? X.sexp[c] : 0; }

// The weights of column c times 2^s (a scratch copy unless s = 0).
const double* weights_for(RowCtx& X, int c, int s) {
  if (s == 0) return X.wts(c);
  const int d = X.col(c).d;
  double* w = X.h->ws.get<double>("w_scaled", d);
  copy(w, X.wts(c), d, X.h->st);
  scale_pow2(w, d, -s, X.h->st);
  return w;
}

// Theta [(bl, chl) x (u, kp)] of the sparse site diagram, 2^weight_exp times
// the true one
void site_diagram(RowCtx& X, int c, const double* Kt, int kp, double* Th) {
  const Column& K_ = X.col(c);
  int chl = X.chl(c), chr = X.chr(c);
  long long m = (long long)K_.nBL() * chl, n = (long long)K_.nU * kp;
  SGTN_CUDA(cudaMemsetAsync(Th, 0, size_t(m * n) * sizeof(double), X.h->st));
  SegGemm a;
  a.name = "site_diagram";
  a.X = X.Ahat[c];
  a.Y = Kt;
  a.O = Th;
  a.p = chl;
  a.q = chr;
  a.s = kp;
  a.xs_i = chr;
  a.xs_k = 1;
  a.xrs = (long long)chl * chr;
  a.ys_k = kp;
  a.ys_j = 1;
  a.yrs = (long long)chr * kp;
  a.os_i = n;
  a.os_j = 1;
  a.ors = (long long)chl * n;
  a.ocs = kp;
  a.seg_ptr = K_.theta.seg_ptr;
  a.vseg_ptr = K_.theta.vseg_ptr;
  a.vfirst = K_.theta.vfirst;
  a.nvseg = K_.theta.nvseg;
  a.seg_or = K_.theta.seg_or;
  a.seg_oc = K_.theta.seg_oc;
  a.xr = K_.theta.xr;
  a.xc = K_.theta.xc;
  a.yr = K_.theta.yr;
  a.yc = K_.theta.yc;
  a.cidx = K_.theta.cidx;
  a.coef = weights_for(X, c, weight_exp(X, c));
  a.nseg = K_.theta.nseg;
  a.nterm = K_.theta.nterm;
  a.x_rows = (long long)K_.nA() * chl;
  a.y_rows = (long long)K_.nK() * chr;
  seg_gemm(a, X.h->st);
}

// Theta for column c with right tensor K ([nBR][chr][kp]); returns scratch pointer
double* theta_of(RowCtx& X, int c, const double* K, int kp) {
  double* Kt = absorb(X, c, K, kp, "ktil");
  const Column& K_ = X.col(c);
  double* Th = X.h->ws.get<double>("theta", size_t(K_.nBL()) * X.chl(c) * K_.nU * kp);
  site_diagram(X, c, Kt, kp, Th);
  return Th;
}

// L env update: Lnext [b][br][chr] from L [a][bl][chl] and phi_c [a][u][b]
double* update_L(RowCtx& X, int c, const double* L, const Ten& phi) {
  sgtn_inst* h = X.h;
  const Column& K_ = X.col(c);
  int chl = X.chl(c), chr = X.chr(c);
  long long nbl = K_.nBL();
  // N[p][b][chl] = sum_a phi[a][u_p][b] L[a][bl_p][chl] for the (u, bl) pairs
  // p that some state reads (far fewer than all u x bl pairs when both the
  // physical and the left bond index are large)
  const int np = K_.lpairs.nseg;
  double* N = h->ws.get<double>("lupd_N", size_t(np) * phi.b * chl);
  {
    SegGemm n;
    n.name = "env_update";
    n.X = phi.p;
    n.p = phi.b;
    n.q = phi.a;
    n.xs_i = 1;
    n.xs_k = (long long)phi.u * phi.b;
    n.xrs = phi.b;
    n.Y = L;
    n.s = chl;
    n.ys_k = nbl * chl;
    n.ys_j = 1;
    n.yrs = chl;
    n.O = N;
    n.os_i = chl;
    n.os_j = 1;
    n.ors = (long long)phi.b * chl;
    n.out_by_seg = 1;
    n.seg_ptr = K_.lpairs.seg_ptr;
    n.xr = K_.lpairs.xr;
    n.xc = K_.lpairs.xc;
    n.yr = K_.lpairs.yr;
    n.yc = K_.lpairs.yc;
    n.nseg = np;
    n.nterm = np;
    seg_gemm(n, h->st);
  }
  // Ltil[(pr,e,pdr)][b][chr] = sum_terms w_x N[pair(u_x, bl)] Ahat[(pd,e,g)]
  double* Lt = h->ws.get<double>("lupd_Lt", size_t(K_.nK()) * phi.b * chr);
  SGTN_CUDA(cudaMemsetAsync(Lt, 0, size_t(K_.nK()) * phi.b * chr * sizeof(double), h->st));
  SegGemm a;
  a.name = "env_update";
  a.X = N;
  a.p = phi.b;
  a.q = chl;
  a.xs_i = chl;
  a.xs_k = 1;
  a.xrs = (long long)phi.b * chl;
  a.xcs = 0;
  a.Y = X.Ahat[c];
  a.s = chr;
  a.ys_k = chr;
  a.ys_j = 1;
  a.yrs = (long long)chl * chr;
  a.O = Lt;
  a.os_i = chr;
  a.os_j = 1;
  a.ors = (long long)phi.b * chr;
  a.seg_ptr = K_.lupd.seg_ptr;
  a.vseg_ptr = K_.lupd.vseg_ptr;
  a.vfirst = K_.lupd.vfirst;
  a.nvseg = K_.lupd.nvseg;
  a.seg_or = K_.lupd.seg_or;
  a.seg_oc = K_.lupd.seg_oc;
  a.xr = K_.lupd_pair;
  a.xc = K_.lupd.xc;
  a.yr = K_.lupd.yr;
  a.yc = K_.lupd.yc;
  a.cidx = K_.lupd.cidx;
  a.coef = weights_for(X, c, (g_compute_f32 && X.lexp) ? X.lexp[c] : 0);   // the scale is not kept
  a.nseg = K_.lupd.nseg;
  a.nterm = K_.lupd.nterm;
  a.x_rows = (long long)np * phi.b;
  a.y_rows = (long long)K_.nA() * chl;
  seg_gemm(a, h->st);
  // Lnext[b][br][chr] = sum_k Wk[k][br] Ltil[k][b][chr]   (batched over b)
  double* Ln = dmalloc((long long)phi.b * K_.nBR() * chr);
  if (g_use_tc && g_compute_f32) {
    // TF32 mode: one product Wk^T [nBR x nK] Ltil [nK x (b, chr)] (large
    // enough for the dense tensor-core GEMM), then (br, b) -> (b, br)
    const long long n = (long long)phi.b * chr;
    double* C = h->ws.get<double>("lupd_C", size_t(K_.nBR()) * n);
    gemm(K_.Wk, true, K_.nBR(), Lt, false, n, C, n, K_.nBR(), int(n), K_.nK(), 1.0, 0, h->st);
    permute3(C, K_.nBR(), phi.b, chr, Ln, h->st);
    return Ln;
  }
  SegGemm g;
  g.name = "env_update";
  g.X = K_.Wk;
  g.p = K_.nBR();
  g.q = K_.nK();
  g.xs_i = 1;
  g.xs_k = K_.nBR();
  g.xrs = 0;
  g.Y = Lt;
  g.s = chr;
  g.ys_k = (long long)phi.b * chr;
  g.ys_j = 1;
  g.yrs = chr;
  g.O = Ln;
  g.os_i = chr;
  g.os_j = 1;
  g.ors = (long long)K_.nBR() * chr;
  g.nseg = phi.b;
  seg_gemm(g, h->st);
  return Ln;
}

// Left-environment update rescaled by a power of two to a norm near 1; in the
// mixed arithmetic its weight exponent (X.lexp) is adapted when the result's
// norm leaves 2^+-100 (at most four retries).
double* update_L_adapt(RowCtx& X, int c, const double* L, const Ten& phi) {
  sgtn_inst* h = X.h;
  const long long n = (long long)phi.b * X.col(c).nBR() * X.chr(c);
  for (int tries = 0;; ++tries) {
    double* Ln = update_L(X, c, L, phi);
    const double v = norm_value(h, Ln, n);
    const int step = (g_compute_f32 && X.lexp && tries < 4) ? exp_step(v) : 0;
    if (step == 0) {
      if (!std::isfinite(v) || !(v > 0.0)) throw SgtnError(-4, "zero or non-finite norm");
      const int e = (int)std::lround(std::log2(v));
      if (e != 0) scale_pow2(Ln, n, e, h->st);
      return Ln;
    }
    X.lexp[c] += step;
    dfree(Ln);
  }
}

// R env update: Rprev[(bl, chl)][a] = Theta_R phi^T
double* update_R(RowCtx& X, int c, const double* ThR, const Ten& phi) {
  const Column& K_ = X.col(c);
  long long m = (long long)K_.nBL() * X.chl(c), n = (long long)X.nout(c) * phi.b;
  double* Rp = dmalloc(m * phi.a);
  gemm(ThR, false, n, phi.p, true, n, Rp, phi.a, int(m), phi.a, int(n), 1.0, 0, X.h->st);
  return Rp;
}

void right_canonical(RowCtx& X, std::vector<Ten>& phi) {
  F64Scope f64;
  sgtn_inst* h = X.h;
  for (int c = (int)phi.size() - 1; c > 0; --c) {
    Ten& t = phi[c];
    SvdOut o = svd(h, t.p, t.a, t.u * t.b, 1 << 30);
    const int k = o.k;
    double* Vt = o.Vt;
    double* Lf = o.US;
    o.Vt = o.US = nullptr;
    o.release();
    Ten& l = phi[c - 1];
    double* nl = dmalloc((long long)l.a * l.u * k);
    gemm(l.p, false, l.b, Lf, false, k, nl, k, l.a * l.u, k, l.b, 1.0, 0, h->st);
    dfree(Lf);
    dfree(l.p);
    l.p = nl;
    l.b = k;
    dfree(t.p);
    t.p = Vt;
    t.a = k;
  }
}

// The site-diagram result Theta [(bl, chl) x (out, kp)], dense or block-sparse
// (one chl x kp block per (bl, u) segment of the column's term table: most
// (bl, u) pairs never occur, so the block form holds far fewer entries).
struct ThetaOp {
  bool bs = false;
  double* dense = nullptr;
  double* blocks = nullptr;
  int m = 0, n = 0, chl = 0, kp = 0, nseg = 0, nbl = 0, nout = 0;
  int s = 0;   // the stored Theta is 2^s times the true one (weight_exp)
};

ThetaOp theta_op(RowCtx& X, int c, const double* K, int kp) {
  ThetaOp T;
  const Column& K_ = X.col(c);
  T.chl = X.chl(c);
  T.kp = kp;
  T.nbl = K_.nBL();
  T.nout = X.nout(c);
  T.m = T.nbl * T.chl;
  T.n = T.nout * kp;
  T.s = weight_exp(X, c);
  sgtn_inst* h = X.h;
  if ((long long)T.m * T.n <= h->bs_min_entries) {
    T.dense = theta_of(X, c, K, kp);
    return T;
  }
  T.bs = true;
  T.nseg = K_.theta.nseg;
  double* Kt = absorb(X, c, K, kp, "ktil");
  T.blocks = h->ws.get<double>("theta_bs", size_t(T.nseg) * T.chl * kp);
  SegGemm a;
  a.name = "site_diagram";
  a.X = X.Ahat[c];
  a.Y = Kt;
  a.O = T.blocks;
  a.p = T.chl;
  a.q = X.chr(c);
  a.s = kp;
  a.xs_i = X.chr(c);
  a.xs_k = 1;
  a.xrs = (long long)T.chl * X.chr(c);
  a.ys_k = kp;
  a.ys_j = 1;
  a.yrs = (long long)X.chr(c) * kp;
  a.os_i = kp;
  a.os_j = 1;
  a.ors = (long long)T.chl * kp;
  a.out_by_seg = 1;
  a.seg_ptr = K_.theta.seg_ptr;
  a.vseg_ptr = K_.theta.vseg_ptr;
  a.vfirst = K_.theta.vfirst;
  a.nvseg = K_.theta.nvseg;
  a.seg_or = K_.theta.seg_or;
  a.seg_oc = K_.theta.seg_oc;
  a.xr = K_.theta.xr;
  a.xc = K_.theta.xc;
  a.yr = K_.theta.yr;
  a.yc = K_.theta.yc;
  a.cidx = K_.theta.cidx;
  a.coef = weights_for(X, c, T.s);
  a.nseg = K_.theta.nseg;
  a.nterm = K_.theta.nterm;
  a.x_rows = (long long)K_.nA() * T.chl;
  a.y_rows = (long long)K_.nK() * X.chr(c);
  seg_gemm(a, h->st);
  return T;
}

// Y (m x s) = Theta Q (Q: n x s)
void theta_mul(RowCtx& X, int c, const ThetaOp& T, const double* Q, int s, double* Y) {
  if (!T.bs) {
    gemm(T.dense, false, T.n, Q, false, s, Y, s, T.m, s, T.n, 1.0, 0, X.h->st);
    return;
  }
  const TermTable& t = X.col(c).bs_rows;
  SGTN_CUDA(cudaMemsetAsync(Y, 0, size_t(T.m) * s * sizeof(double), X.h->st));
  SegGemm a;
  a.name = "theta_mul";
  a.X = T.blocks;
  a.p = T.chl;
  a.q = T.kp;
  a.xs_i = T.kp;
  a.xs_k = 1;
  a.xrs = (long long)T.chl * T.kp;
  a.Y = Q;
  a.s = s;
  a.ys_k = s;
  a.ys_j = 1;
  a.yrs = (long long)T.kp * s;
  a.O = Y;
  a.os_i = s;
  a.os_j = 1;
  a.ors = (long long)T.chl * s;
  a.seg_ptr = t.seg_ptr;
  a.vseg_ptr = t.vseg_ptr;
  a.vfirst = t.vfirst;
  a.nvseg = t.nvseg;
  a.seg_or = t.seg_or;
  a.seg_oc = t.seg_oc;
  a.xr = t.xr;
  a.xc = t.xc;
  a.yr = t.yr;
  a.yc = t.yc;
  a.nseg = t.nseg;
  a.nterm = t.nterm;
  seg_gemm(a, X.h->st);
}

// Z (n x s) = Theta^T Y (Y: m x s)
void theta_tmul(RowCtx& X, int c, const ThetaOp& T, const double* Y, int s, double* Z) {
  if (!T.bs) {
    gemm(T.dense, true, T.n, Y, false, s, Z, s, T.n, s, T.m, 1.0, 0, X.h->st);
    return;
  }
  const TermTable& t = X.col(c).bs_cols;
  SGTN_CUDA(cudaMemsetAsync(Z, 0, size_t(T.n) * s * sizeof(double), X.h->st));
  SegGemm a;
  a.name = "theta_mul";
  a.X = T.blocks;
  a.p = T.kp;
  a.q = T.chl;
  a.xs_i = 1;
  a.xs_k = T.kp;
  a.xrs = (long long)T.chl * T.kp;
  a.Y = Y;
  a.s = s;
  a.ys_k = s;
  a.ys_j = 1;
  a.yrs = (long long)T.chl * s;
  a.O = Z;
  a.os_i = s;
  a.os_j = 1;
  a.ors = (long long)T.kp * s;
  a.seg_ptr = t.seg_ptr;
  a.vseg_ptr = t.vseg_ptr;
  a.vfirst = t.vfirst;
  a.nvseg = t.nvseg;
  a.seg_or = t.seg_or;
  a.seg_oc = t.seg_oc;
  a.xr = t.xr;
  a.xc = t.xc;
  a.yr = t.yr;
  a.yc = t.yc;
  a.nseg = t.nseg;
  a.nterm = t.nterm;
  seg_gemm(a, X.h->st);
}

// t (a x n) = L_mat (a x m) Theta
double* theta_left(RowCtx& X, int c, const ThetaOp& T, const double* L, int a_dim) {
  double* t = dmalloc((long long)a_dim * T.n);
  if (!T.bs) {
    gemm(L, false, T.m, T.dense, false, T.n, t, T.n, a_dim, T.n, T.m, 1.0, 0, X.h->st);
    return t;
  }
  const TermTable& tt = X.col(c).bs_cols;
  SGTN_CUDA(cudaMemsetAsync(t, 0, size_t(a_dim) * T.n * sizeof(double), X.h->st));
  SegGemm a;
  a.name = "theta_env";
  a.X = L;
  a.p = a_dim;
  a.q = T.chl;
  a.xs_i = T.m;
  a.xs_k = 1;
  a.xcs = T.chl;
  a.Y = T.blocks;
  a.s = T.kp;
  a.ys_k = T.kp;
  a.ys_j = 1;
  a.ycs = (long long)T.chl * T.kp;
  a.O = t;
  a.os_i = T.n;
  a.os_j = 1;
  a.ors = T.kp;
  a.seg_ptr = tt.seg_ptr;
  a.vseg_ptr = tt.vseg_ptr;
  a.vfirst = tt.vfirst;
  a.nvseg = tt.nvseg;
  a.seg_or = tt.seg_or;
  a.seg_oc = tt.seg_oc;
  a.xr = tt.xr;
  a.xc = tt.xc;
  a.yr = tt.yr;
  a.yc = tt.yc;
  a.nseg = tt.nseg;
  a.nterm = tt.nterm;
  seg_gemm(a, X.h->st);
  return t;
}

// R (m x a) = Theta phi_mat^T  with phi [a][out][b]
double* theta_right(RowCtx& X, int c, const ThetaOp& T, const Ten& phi) {
  if (!T.bs) return update_R(X, c, T.dense, phi);
  double* Rp = dmalloc((long long)T.m * phi.a);
  const TermTable& tt = X.col(c).bs_rows;
  SGTN_CUDA(cudaMemsetAsync(Rp, 0, size_t(T.m) * phi.a * sizeof(double), X.h->st));
  SegGemm a;
  a.name = "theta_env";
  a.X = T.blocks;
  a.p = T.chl;
  a.q = T.kp;
  a.xs_i = T.kp;
  a.xs_k = 1;
  a.xrs = (long long)T.chl * T.kp;
  a.Y = phi.p;
  a.s = phi.a;
  a.ys_k = 1;
  a.ys_j = T.n;
  a.yrs = T.kp;
  a.O = Rp;
  a.os_i = phi.a;
  a.os_j = 1;
  a.ors = (long long)T.chl * phi.a;
  a.seg_ptr = tt.seg_ptr;
  a.vseg_ptr = tt.vseg_ptr;
  a.vfirst = tt.vfirst;
  a.nvseg = tt.nvseg;
  a.seg_or = tt.seg_or;
  a.seg_oc = tt.seg_oc;
  a.xr = tt.xr;
  a.xc = tt.xc;
  a.yr = tt.yr;
  a.yc = tt.yc;
  a.nseg = tt.nseg;
  a.nterm = tt.nterm;
  seg_gemm(a, X.h->st);
  return Rp;
}

SvdOut theta_svd(RowCtx& X, int c, const ThetaOp& T, int cap) {
  sgtn_inst* h = X.h;
  if (!T.bs) return svd(h, T.dense, T.m, T.n, cap);
  int p = std::min(T.m, T.n);
  if (p <= h->dense_svd_max || cap >= p) {
    double* D = h->ws.get<double>("theta_dense_of_bs", size_t(T.m) * T.n);
    SGTN_CUDA(cudaMemsetAsync(D, 0, size_t(T.m) * T.n * sizeof(double), h->st));
    const Column& K_ = X.col(c);
    scatter_blocks(T.blocks, T.nseg, T.chl, T.kp, K_.theta.seg_or, K_.theta.seg_oc, D, T.n, h->st);
    return svd(h, D, T.m, T.n, cap);
  }
  MatFn mul = [&](const double* Q, int s, double* Y) { theta_mul(X, c, T, Q, s, Y); };
  MatFn tmul = [&](const double* Y, int s, double* Z) { theta_tmul(X, c, T, Y, s, Z); };
  return profiled(h, "", T.m, T.n, [&] { return svd_subspace_op(h, T.m, T.n, cap, mul, tmul); });
}

// Right environments of a row step, kept across the zipper's stages: R[c] is
// the environment of columns c+1..C-1 at bond (c, c+1), stored
// [(bl, chl) of column c+1] x [left bond of phi[c+1]] (R[C-1] = 1), and its
// value is exp(lg[c]) times the stored one (environments are rescaled by
// powers of two: they would leave the floating-point range).  The zipper's
// connecting tensor after column c is R[c-1].
struct RightEnvs {
  std::vector<double*> R;
  std::vector<double> lg;
  explicit RightEnvs(int C) : R(C, nullptr), lg(C, 0.0) {}
  RightEnvs(const RightEnvs&) = delete;
  RightEnvs& operator=(const RightEnvs&) = delete;
  ~RightEnvs() {
    for (auto& p : R) dfree(p);
  }
  void set(int c, double* p, double l) {
    if (R[c] != p) dfree(R[c]);
    R[c] = p;
    lg[c] = l;
  }
};

// One sweep of one-site overlap maximisation (Fig. 8d) over columns c0..e of
// phi, left to right and back.  The target is the MPO-MPS product of columns
// c0..C-1 with its left bond open when c0 > 0 (the instantaneous stage of the
// zipper); phi must be right-canonical on c0..C-1, Lc0 [phi[c0].a x (bl, chl)
// of column c0] is the left environment at c0 (taken over, freed here) and
// RE.R[c0..e] must hold the environments of the current phi.  Each update is
// the exact maximiser given the other tensors, made orthonormal by a
// CholeskyQR pass and a polar correction where the truncated SVD would keep
// every direction (orth_qr: only the span matters, the next update projects
// onto it again), else by that SVD.
// Afterwards phi[c0..e] are right-canonical and RE.R[c0-1..e-1] refreshed:
// for c0 > 0, RE.R[c0-1] is the new connecting tensor (the optimal centre of
// the stage); for c0 = 0 the centre stays in phi[0] (unnormalised) and the
// log-scale of its right environment is returned.
double sweep_range(RowCtx& X, std::vector<Ten>& phi, int c0, int e, double* Lc0, RightEnvs& RE) {
  sgtn_inst* h = X.h;
  TagScope tag("sweep");
  const int C = (int)phi.size();
  std::vector<double*> Lenv(C, nullptr);
  Lenv[c0] = Lc0;
  for (int c = c0; c <= e; ++c) {
    ThetaOp T = theta_op(X, c, RE.R[c], phi[c].b);
    const int a = phi[c].a;
    double* t = theta_left(X, c, T, Lenv[c], a);
    dfree(phi[c].p);
    phi[c].p = t;
    phi[c].u = X.nout(c);
    if (c < e) {
      const int m = a * X.nout(c);
      double* Q = h->sweep_qr ? dmalloc((long long)m * phi[c].b) : nullptr;
      if (Q && orth_qr(h, t, m, phi[c].b, false, Q)) {
        ++h->sweep_qr_count;
        dfree(phi[c].p);
        phi[c].p = Q;
      } else {
        dfree(Q);
        ++h->sweep_svd_count;
        SvdOut o = svd(h, t, m, phi[c].b, 1 << 30);
        Q = left_factor(h, o, m);
        dfree(phi[c].p);
        phi[c].p = Q;
        phi[c].b = o.k;
        o.release();
      }
      Lenv[c + 1] = update_L_adapt(X, c, Lenv[c], phi[c]);
      // the next site's left bond is now o.k; its right bond is unchanged
      phi[c + 1].a = phi[c].b;
    }
  }
  double rc_log = RE.lg[e];
  int s_c0 = 0;
  for (int c = e; c >= c0; --c) {
    ThetaOp T = theta_op(X, c, RE.R[c], phi[c].b);
    if (c == c0) s_c0 = T.s;
    const int a = phi[c].a;
    const long long n = (long long)X.nout(c) * phi[c].b;
    double* t = theta_left(X, c, T, Lenv[c], a);
    dfree(phi[c].p);
    phi[c].p = t;
    if (c > 0) {
      double* Q = h->sweep_qr ? dmalloc((long long)a * n) : nullptr;
      if (Q && orth_qr(h, t, a, int(n), true, Q)) {
        ++h->sweep_qr_count;
        dfree(phi[c].p);
        phi[c].p = Q;
      } else {
        dfree(Q);
        ++h->sweep_svd_count;
        SvdOut o = svd(h, t, a, int(n), 1 << 30);
        dfree(phi[c].p);
        phi[c].p = o.Vt;
        o.Vt = nullptr;
        phi[c].a = o.k;
        o.release();
      }
      double* Rn = theta_right(X, c, T, phi[c]);
      rescale_pow2(h, Rn, (long long)X.col(c).nBL() * X.chl(c) * phi[c].a, rc_log);
      rc_log -= T.s * kLn2;
      RE.set(c - 1, Rn, rc_log);
      if (c > c0) phi[c - 1].b = phi[c].a;
    }
  }
  for (auto& p : Lenv) dfree(p);
  // for c0 = 0 the centre phi[0] came from column 0's (scaled) Theta
  if (c0 == 0) rc_log -= s_c0 * kLn2;
  return rc_log;
}

// One full left-right-left sweep (c0 = 0, e = C-1) from freshly built right
// environments; returns the log-scale of the centre phi[0].
double variational_sweep(RowCtx& X, std::vector<Ten>& phi, bool canonical) {
  sgtn_inst* h = X.h;
  const int C = (int)phi.size();
  // phi coming from the zipper or from a previous sweep is already right-
  // canonical (orthonormal rows right of a centre at column 0): bringing it
  // there again would only change the gauge
  if (!canonical) right_canonical(X, phi);
  RightEnvs RE(C);
  RE.R[C - 1] = dmalloc(1);
  fill(RE.R[C - 1], 1, 1.0, h->st);
  double lg = 0.0;
  for (int c = C - 1; c > 0; --c) {
    ThetaOp T = theta_op(X, c, RE.R[c], phi[c].b);
    double* Rn = theta_right(X, c, T, phi[c]);
    rescale_pow2(h, Rn, (long long)X.col(c).nBL() * X.chl(c) * phi[c].a, lg);
    lg -= T.s * kLn2;
    RE.set(c - 1, Rn, lg);
  }
  double* L0 = dmalloc(1);
  fill(L0, 1, 1.0, h->st);
  return sweep_range(X, phi, 0, C - 1, L0, RE);
}

// cut a right-canonical phi (centre 0) to bond chi; returns worst retained ratio
double svd_cut(RowCtx& X, std::vector<Ten>& phi, int chi) {
  F64Scope f64;
  TagScope tag("cut");
  sgtn_inst* h = X.h;
  double worst = 0.0;
  for (int c = 0; c + 1 < (int)phi.size(); ++c) {
    Ten& t = phi[c];
    SvdOut o = svd(h, t.p, t.a * t.u, t.b, chi);
    worst = std::max(worst, o.sig.back() / o.sig.front());
    double* Q = left_factor(h, o, t.a * t.u);
    double* Rm = right_factor(h, o, t.b);
    dfree(t.p);
    t.p = Q;
    Ten& n = phi[c + 1];
    double* nn = dmalloc((long long)o.k * n.u * n.b);
    gemm(Rm, false, t.b, n.p, false, (long long)n.u * n.b, nn, (long long)n.u * n.b, o.k, n.u * n.b, t.b, 1.0, 0,
         h->st);
    dfree(Rm);
    dfree(n.p);
    n.p = nn;
    n.a = o.k;
    t.b = o.k;
    o.release();
  }
  return worst;
}

void left_canonical(sgtn_inst* h, MPS& A) {
  F64Scope f64;
  TagScope tag("left_canonical");
  const int C = A.C;
  for (int c = 0; c + 1 < C; ++c) {
    int s = A.phys[c], l = A.bond[c], r = A.bond[c + 1];
    SvdOut o = svd(h, A.t[c], s * l, r, 1 << 30);
    double* Q = left_factor(h, o, s * l);
    double* Rm = right_factor(h, o, r);
    dfree(A.t[c]);
    A.t[c] = Q;
    int s2 = A.phys[c + 1], r2 = A.bond[c + 2];
    double* nn = dmalloc((long long)s2 * o.k * r2);
    // nn[s][k][r2] = sum_r Rm[k][r] A[s][r][r2]   (batched over s)
    SegGemm g;
    g.name = "mps_absorb";
    g.X = Rm;
    g.p = o.k;
    g.q = r;
    g.xs_i = r;
    g.xs_k = 1;
    g.xrs = 0;
    g.Y = A.t[c + 1];
    g.s = r2;
    g.ys_k = r2;
    g.ys_j = 1;
    g.yrs = (long long)r * r2;
    g.O = nn;
    g.os_i = r2;
    g.os_j = 1;
    g.ors = (long long)o.k * r2;
    g.nseg = s2;
    seg_gemm(g, h->st);
    dfree(Rm);
    dfree(A.t[c + 1]);
    A.t[c + 1] = nn;
    A.bond[c + 1] = o.k;
    o.release();
  }
  long long nl = (long long)A.phys[C - 1] * A.bond[C - 1] * A.bond[C];
  normalise(h, A.t[C - 1], nl, A.lognorm);
}

void compute_ahat(RowCtx& X) {
  const int C = X.h->M.C;
  X.Ahat.assign(C, nullptr);
  for (int c = 0; c < C; ++c) {
    const Column& K_ = X.col(c);
    long long blk = (long long)X.chl(c) * X.chr(c);
    X.Ahat[c] = dmalloc(K_.nA() * blk);
    gemm(K_.Wa, false, K_.nSig, X.A->t[c], false, blk, X.Ahat[c], blk, K_.nA(), int(blk), K_.nSig, 1.0, 0,
         X.h->st);
  }
}

// Sign of a 1x1 device tensor, folded into phi[0] when negative (the
// zipper's last connecting tensor carries the overall sign of the row).
void absorb_sign(sgtn_inst* h, const double* K, Ten& phi0) {
  double kv = 0;
  SGTN_CUDA(cudaMemcpyAsync(&kv, K, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  if (kv < 0) {
    double* m1 = h->ws.get<double>("minus_one", 1);
    fill(m1, 1, -1.0, h->st);
    scale_by_inv(phi0.p, phi0.n(), m1, h->st);
  }
}

// out ~ T A (T = the row MPO of X); A is left-canonicalised in place.
// Sec. III.B "Variational zipper algorithm": right to left, each zipper step
// (SVD truncation of the dashed-box tensor to 2 chi values, Fig. 8c) is
// followed by a one-site sweep of the instantaneous stage over the columns
// built so far, or over the h->zipper_window columns next to the zipper
// centre (Fig. 8d); then the cut to chi and n_sweeps full sweeps at chi.
void row_step_ctx(RowCtx& X, MPS& A, int chi, int n_sweeps, MPS& out, double& worst) {
  sgtn_inst* h = X.h;
  const int C = h->M.C;
  left_canonical(h, A);
  X.A = &A;
  compute_ahat(X);
  std::vector<Ten> phi(C);
  RightEnvs RE(C);
  RE.R[C - 1] = dmalloc(1);
  fill(RE.R[C - 1], 1, 1.0, h->st);
  const int w = h->zipper_window;
  double ln = A.lognorm;
  for (int c = C - 1; c >= 0; --c) {
    const Column& K_ = X.col(c);
    const int kp = c == C - 1 ? 1 : phi[c + 1].a;
    const int m = K_.nBL() * X.chl(c);
    SvdOut o;
    int ts = 0;
    {
      TagScope tag("zipper");
      // in the mixed arithmetic the weights' exponent is adapted when the
      // largest singular value of Theta leaves 2^+-100 (a result that left
      // FP32's range entirely raises the weights by 2^100)
      for (int tries = 0;; ++tries) {
        ThetaOp T = theta_op(X, c, RE.R[c], kp);
        ts = T.s;
        const bool adapt = g_compute_f32 && X.sexp && tries < 4;
        try {
          o = theta_svd(X, c, T, 2 * chi);
        } catch (const SgtnError& err) {
          if (!adapt || err.code != -4) throw;
          X.sexp[c] += 100;
          continue;
        }
        if (!adapt || !(o.sig[0] > 0.0) || !std::isfinite(o.sig[0])) break;
        const int ex = std::ilogb(o.sig[0]);
        if (ex >= -100 && ex <= 100) break;
        X.sexp[c] -= ex;
        o.release();
      }
    }
    phi[c].p = o.Vt;
    o.Vt = nullptr;
    phi[c].a = o.k;
    phi[c].u = X.nout(c);
    phi[c].b = kp;
    const int e = w <= 0 ? C - 1 : std::min(C - 1, c + w - 1);
    if (e > c) {
      // the centre moves from the connecting tensor K = U S onto phi[c]: U^T
      // is the left environment of column c (for c = 0, K is 1x1 and the
      // sweep recomputes the centre from scratch)
      double* L0 = nullptr;
      if (c > 0) {
        double* Q = left_factor(h, o, m);
        L0 = dmalloc((long long)o.k * m);
        permute3(Q, m, o.k, 1, L0, h->st);
        dfree(Q);
      } else {
        L0 = dmalloc(1);
        fill(L0, 1, 1.0, h->st);
      }
      o.release();
      const double lg = sweep_range(X, phi, c, e, L0, RE);
      // the stage's centre is computed from the target itself: its scale is
      // relative to the input MPS alone
      if (c > 0) {
        ln = A.lognorm + RE.lg[c - 1];
        normalise(h, RE.R[c - 1], (long long)m * phi[c].a, ln);
        RE.lg[c - 1] = ln - A.lognorm;
      } else {
        ln = A.lognorm + lg;
        normalise(h, phi[0].p, phi[0].n(), ln);
      }
    } else {
      double* K = o.US;
      o.US = nullptr;
      o.release();
      normalise(h, K, (long long)m * phi[c].a, ln);
      ln -= ts * kLn2;
      if (c > 0) {
        RE.set(c - 1, K, ln - A.lognorm);
      } else {
        absorb_sign(h, K, phi[0]);
        dfree(K);
      }
    }
  }
  worst = std::max(worst, svd_cut(X, phi, chi));
  normalise(h, phi[C - 1].p, phi[C - 1].n(), ln);
  for (int s = 0; s < n_sweeps; ++s) {
    // optionally the sweeps after the cut in FP64 also in a mixed contraction:
    // they converge the MPS toward the fixed point of the FP64 target
    std::unique_ptr<F64Scope> f64;
    if (h->f64_final_sweeps) f64.reset(new F64Scope());
    double extra = variational_sweep(X, phi, s > 0);   // svd_cut leaves phi left-canonical
    ln = A.lognorm + extra;
    normalise(h, phi[0].p, phi[0].n(), ln);
  }
  for (double*& p : X.Ahat) dfree(p);
  X.Ahat.clear();
  // store as [phys][bond_l][bond_r]
  free_mps(out);
  out.C = C;
  out.phys.assign(C, 1);
  out.bond.assign(C + 1, 1);
  out.t.assign(C, nullptr);
  for (int c = 0; c < C; ++c) {
    out.phys[c] = phi[c].u;
    out.bond[c] = phi[c].a;
    out.bond[c + 1] = phi[c].b;
    out.t[c] = dmalloc(phi[c].n());
    permute3(phi[c].p, phi[c].a, phi[c].u, phi[c].b, out.t[c], h->st);
    dfree(phi[c].p);
  }
  out.lognorm = ln;
  out.valid = true;
  h->check();
}

// psi_{r-1} ~ T_r psi_r (sparse projector form)
void row_step(sgtn_inst* h, int r, int chi, int n_sweeps, MPS& out, double& worst) {
  if (std::getenv("SGTN_TRACE")) fprintf(stderr, "[sgtn] row step %d\n", r);
  RowCtx X;
  X.h = h;
  X.r = r;
  X.sexp = &h->theta_exp[size_t(r) * h->M.C];
  X.lexp = &h->lenv_exp[size_t(r) * h->M.C];
  row_step_ctx(X, h->psi[r], chi, n_sweeps, out, worst);
}

double top_overlap(sgtn_inst* h) {
  F64Scope f64;   // one row: FP64, no weight scaling
  const int C = h->M.C;
  MPS& A = h->psi[0];
  RowCtx X;
  X.h = h;
  X.r = 0;
  X.A = &A;
  compute_ahat(X);
  double ln = A.lognorm;
  double* Rc = dmalloc(1);
  fill(Rc, 1, 1.0, h->st);
  for (int c = C - 1; c >= 0; --c) {
    const Column& K_ = X.col(c);
    double* Th = theta_of(X, c, Rc, 1);
    long long m = (long long)K_.nBL() * X.chl(c);
    double* Rn = dmalloc(m);
    copy(Rn, Th, m, h->st);  // nU = 1 in the top row
    dfree(Rc);
    Rc = Rn;
    if (c > 0) normalise(h, Rc, m, ln);
  }
  double v = 0;
  SGTN_CUDA(cudaMemcpyAsync(&v, Rc, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  dfree(Rc);
  for (double*& p : X.Ahat) dfree(p);
  if (!std::isfinite(v)) throw SgtnError(-4, "non-finite top-row overlap");
  // an approximate psi_0 (negative entries, Sec. V) can give a non-positive
  // overlap: log Z is then undefined (NaN); the boundary MPSs stay usable for
  // the branch step, whose scores are clamped at 0
  if (!(v > 0.0)) return std::nan("");
  return ln + std::log(v);
}

}  // namespace detail

using namespace detail;

void contract_boundary(sgtn_inst* h, int chi, int n_sweeps) {
  const int R = h->M.R, C = h->M.C;
  for (auto& m : h->psi) free_mps(m);
  h->psi.assign(R, MPS());
  MPS& last = h->psi[R - 1];
  last.C = C;
  last.phys.assign(C, 1);
  last.bond.assign(C + 1, 1);
  last.t.assign(C, nullptr);
  for (int c = 0; c < C; ++c) {
    last.t[c] = dmalloc(1);
    fill(last.t[c], 1, 1.0, h->st);
  }
  last.lognorm = 0.0;
  last.valid = true;
  double worst = 0.0;
  h->unconverged_cuts = 0;
  for (int r = R - 1; r >= 1; --r) row_step(h, r, chi, n_sweeps, h->psi[r - 1], worst);
  h->logz = h->log_offset + top_overlap(h);
  if (prof_on()) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& kv : g_prof)
      fprintf(stderr, "[sgtn] svd %-22s calls %6lld  %9.1f ms  iters %6lld  max %d x %d\n", kv.first.c_str(),
              kv.second.calls, kv.second.ms, kv.second.iters, kv.second.max_m, kv.second.max_n);
    g_prof.clear();
  }
  h->worst_sv = worst;
  h->chi = chi;
  h->n_sweeps = n_sweeps;
  h->boundary_ok = true;
}

}  // namespace sgtn
