// The opaque handle behind sgtn_h (internal).
#pragma once
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "kern.h"
#include "model.h"

#define SGTN_CUDA(x)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess)                                                                        \
      throw SgtnError(e_ == cudaErrorMemoryAllocation ? -3 : -6,                                  \
                      std::string(#x) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

namespace sgtn {

struct DSite {
  int d = 0;
  int64_t* E = nullptr;
  double* w = nullptr;
  int32_t* cls[8] = {};                   // class toward each direction, per state
  int32_t *lam_x = nullptr, *u_x = nullptr, *xk_x = nullptr;
  int32_t *U_u = nullptr, *U_ul = nullptr, *U_ur = nullptr, *Lam_l = nullptr, *Lam_dl = nullptr;
};

// Named growable device scratch buffers.
struct Scratch {
  std::map<std::string, std::pair<void*, size_t>> bufs;
  void* get(const std::string& name, size_t bytes) {
    auto& b = bufs[name];
    if (b.second < bytes) {
      if (b.first) cudaFree(b.first);
      b.first = nullptr;
      size_t nb = bytes + bytes / 4 + 256;
      SGTN_CUDA(lib_malloc(&b.first, nb));
      b.second = nb;
    }
    return b.first;
  }
  template <class T>
  T* get(const std::string& name, size_t count) {
    return static_cast<T*>(get(name, count * sizeof(T)));
  }
  void release() {
    for (auto& kv : bufs)
      if (kv.second.first) cudaFree(kv.second.first);
    bufs.clear();
  }
  size_t total() const {
    size_t t = 0;
    for (auto& kv : bufs) t += kv.second.second;
    return t;
  }
};

}  // namespace sgtn

struct sgtn_inst {
  int device = 0;
  cudaStream_t st = nullptr;
  std::string err;
  sgtn::Model M;
  std::vector<sgtn::DSite> ds;
  std::vector<int64_t*> dE;               // [site*4+k] compressed energies
  std::vector<double*> dB;                // [site*4+k] bond factors exp(-beta (Ebar - min))
  std::vector<sgtn::Column> cols;         // [r*C + c]
  sgtn::GradTables grad;                  // the gradient path's tables (built on first use)
  std::vector<int> theta_exp;             // [r*C + c] weight exponents of the mixed contractions
  std::vector<int> lenv_exp;              // [r*C + c] the same for the left-environment updates
  std::vector<void*> allocs;              // static allocations
  double beta = 0.0;
  bool beta_set = false;
  double log_offset = 0.0;
  std::vector<sgtn::MPS> psi;             // psi[r] covers rows r+1..R-1
  int chi = 0, precision = 0, n_sweeps = 0;
  int zipper_window = 0;                  // columns swept after each zipper step; 0: all built so far
  bool f64_final_sweeps = false;          // the sweeps after the cut in FP64 in a mixed contraction
  bool sweep_qr = true;                   // sweep orthonormalisations by CholeskyQR where the rank rule keeps all
  int search_precision = -1;              // conditionals / branch step / search; -1: as the boundary
  bool boundary_ok = false;
  double logz = 0.0, worst_sv = 0.0;
  sgtn::Scratch ws;
  int32_t* iota = nullptr;                // 0..iota_n-1
  int dense_svd_max = 320;                // exact Jacobi up to this many vectors, subspace iteration above
  long long bs_min_entries = 1ll << 22;   // keep Theta block-sparse when dense would exceed this
  int unconverged_cuts = 0;               // iterative truncations stopped at their cap (no gap)
  long long sweep_qr_count = 0, sweep_svd_count = 0;   // sweep orthonormalisations by each route
  int32_t *d_ei = nullptr, *d_ej = nullptr, *d_jn = nullptr, *d_hn = nullptr;   // edges for energies
  int iota_n = 0;

  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = nullptr;
    size_t n = v.empty() ? 1 : v.size();
    SGTN_CUDA(sgtn::lib_malloc(&p, n * sizeof(T)));
    allocs.push_back(p);
    if (!v.empty()) SGTN_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return p;
  }
  template <class T>
  T* dalloc(size_t n) {
    T* p = nullptr;
    SGTN_CUDA(sgtn::lib_malloc(&p, (n ? n : 1) * sizeof(T)));
    allocs.push_back(p);
    return p;
  }
  void sync() { SGTN_CUDA(cudaStreamSynchronize(st)); }
  void check() { SGTN_CUDA(cudaGetLastError()); }
};

namespace sgtn {
// setup.cu
void setup_device(sgtn_inst* h);
void build_column_tables(sgtn_inst* h, Column& K, const std::vector<int32_t>& lam, const std::vector<int32_t>& u,
                         const std::vector<int32_t>& pd, const std::vector<int32_t>& pr,
                         const std::vector<int32_t>& pdr);
void build_pair_table(sgtn_inst* h, TermTable& tt, const std::vector<int32_t>& xr, const std::vector<int32_t>& yr);
void set_beta_device(sgtn_inst* h, double beta);
void free_mps(MPS& m);
// boundary.cu
void contract_boundary(sgtn_inst* h, int chi, int n_sweeps);
// branch.cu
void conditionals(sgtn_inst* h, int step, int count, const int32_t* configs, double* out_p);
void branch_step(sgtn_inst* h, int step, int M, int in_count, const int32_t* in_configs, const double* in_logp,
                 int32_t* out_configs, double* out_logp, int32_t* out_count, double* io_pd);
// Droplets of Fig. 4 (the excitation bookkeeping of the merges)
struct DropletOpts {
  long long max_dE = 0;   // energy window (numerator over denom)
  int min_hamming = 0;    // kept droplets differ pairwise in more flips than this
};
struct Drop {
  long long dE = 0;
  std::vector<int32_t> flips;   // spin ids, increasing
};
void search(sgtn_inst* h, int M, int n_out, int8_t* out_spins, int64_t* out_energy, double* out_logp, double* out_pd,
            int32_t* out_count,
            const DropletOpts* dopt = nullptr, std::vector<Drop>* dout = nullptr);
void energies(sgtn_inst* h, int n, const int8_t* spins, int64_t* out);
void lbp(sgtn_inst* h, int n_iter, int k, int32_t* out_index, double* out_marginal, int32_t* out_count,
         double* out_change);
void logz_grad(sgtn_inst* h, double* dJ, double* dh, double* dbeta);
size_t scores_scratch_bytes(sgtn_inst* h, int step, int K);
void conditionals_arena(sgtn_inst* h, int step, int count, const int32_t* configs, double* out_p, void* arena,
                        size_t cap);
}  // namespace sgtn

namespace sgtn {
// Device tensors of the contraction (MPS sites, SVD factors, environments) come
// from a cache: a freed block is kept, keyed by its stream and rounded size,
// and handed to the next request of that size on the same stream (stream
// order makes the reuse safe), so a row step does not call cudaMalloc /
// cudaFree -- which synchronises the device -- per tensor.  pool_set_stream
// names the stream of the calling thread's handle; pool_trim frees a stream's
// cached blocks with cudaFree (at sgtn_destroy).
void pool_set_stream(cudaStream_t st);
void* pool_alloc(size_t bytes);
void pool_free(void* p);
void pool_trim(cudaStream_t st);

// Arithmetic of the contractions issued inside one API call: FP32 (plus
// tcgen05 tensor cores for large dense GEMMs with TF32) or FP64, from the
// precision of the last contract_boundary, or, for the conditionals, branch
// step and search, from the search precision when one was set.  Values:
// 0 FP64, 1 TF32, 3 FP32 (sgtn_precision).
struct PrecisionScope {
  PrecisionScope(const sgtn_inst* h, bool search) {
    const int p = (search && h->search_precision >= 0) ? h->search_precision : h->precision;
    g_compute_f32 = p == 3 || p == 1 || p == 2;
    g_use_tc = p == 1 || p == 2;
    g_tc_bf16 = p == 2;
  }
  ~PrecisionScope() {
    g_compute_f32 = false;
    g_use_tc = false;
    g_tc_bf16 = false;
  }
};
}  // namespace sgtn
