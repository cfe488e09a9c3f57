// C ABI of the sgtn library: argument checks, error capture, dispatch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/sgtn.h"
#include "handle.h"

namespace sgtn {

namespace {
// H = sum j s_i s_j + sum h s_i, exact in int64, one block per configuration
__global__ void energy_kernel(int N, long long nE, const int8_t* spins, const int32_t* ei, const int32_t* ej,
                              const int32_t* jn, const int32_t* hn, long long* out) {
  const int8_t* s = spins + (long long)blockIdx.x * N;
  long long a = 0;
  for (long long e = threadIdx.x; e < nE; e += blockDim.x) a += (long long)jn[e] * s[ei[e]] * s[ej[e]];
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += (long long)hn[i] * s[i];
  __shared__ long long red[32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}
}  // namespace

void energies(sgtn_inst* h, int n, const int8_t* spins, int64_t* out) {
  if (n <= 0) return;
  for (long long i = 0; i < (long long)n * h->M.N; ++i)
    if (spins[i] != 1 && spins[i] != -1) throw SgtnError(-1, "spins must be +1 or -1");
  static_assert(sizeof(long long) == sizeof(int64_t), "int64");
  int8_t* ds = nullptr;
  long long* dout = nullptr;
  SGTN_CUDA(lib_malloc(&ds, size_t(n) * h->M.N));
  SGTN_CUDA(lib_malloc(&dout, size_t(n) * sizeof(long long)));
  SGTN_CUDA(cudaMemcpyAsync(ds, spins, size_t(n) * h->M.N, cudaMemcpyHostToDevice, h->st));
  if (!h->d_ei) {
    h->d_ei = h->M.ei.empty() ? nullptr : h->upload(h->M.ei);
    h->d_ej = h->M.ej.empty() ? nullptr : h->upload(h->M.ej);
    h->d_jn = h->M.jn.empty() ? nullptr : h->upload(h->M.jn);
    h->d_hn = h->upload(h->M.hn);
  }
  const int32_t *ei = h->d_ei, *ej = h->d_ej, *jn = h->d_jn, *hn = h->d_hn;
  energy_kernel<<<n, 256, 0, h->st>>>(h->M.N, (long long)h->M.ei.size(), ds, ei, ej, jn, hn, dout);
  ++g_count.launches;
  h->check();
  SGTN_CUDA(cudaMemcpyAsync(out, dout, size_t(n) * sizeof(long long), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  cudaFree(ds);
  cudaFree(dout);
}

}  // namespace sgtn

using namespace sgtn;

namespace {
// live handles per stream: a stream's scratch is released with its last handle
std::mutex g_streams_mu;
std::map<cudaStream_t, int> g_stream_users;

template <class F>
int guarded(sgtn_h h, F&& f) {
  if (!h) return SGTN_ERR_ARG;
  try {
    SGTN_CUDA(cudaSetDevice(h->device));
    pool_set_stream(h->st);
    f();
    h->err.clear();
    return SGTN_OK;
  } catch (const SgtnError& e) {
    h->err = e.what();
    cudaGetLastError();
    return e.code;
  } catch (const std::exception& e) {
    h->err = e.what();
    return SGTN_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

int sgtn_build_instance(int32_t n_spins, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* j_num,
                        const int32_t* h_num, int32_t denom, const int32_t* site_of_spin, int32_t rows, int32_t cols,
                        const int64_t* state_offsets, const int64_t* states, void* stream, sgtn_h* out) {
  if (!out) return SGTN_ERR_ARG;
  *out = nullptr;
  sgtn_inst* h = new sgtn_inst();
  cudaGetDevice(&h->device);
  h->st = static_cast<cudaStream_t>(stream);
  {
    std::lock_guard<std::mutex> lk(g_streams_mu);
    ++g_stream_users[h->st];
  }
  if (const char* e = std::getenv("SGTN_DENSE_SVD_MAX")) h->dense_svd_max = std::max(1, std::atoi(e));
  if (const char* e = std::getenv("SGTN_BS_MIN_ENTRIES")) h->bs_min_entries = std::max(0ll, std::atoll(e));
  std::string e = h->M.build(n_spins, n_edges, ei, ej, j_num, h_num, denom, site_of_spin, rows, cols, state_offsets,
                             states);
  if (!e.empty()) {
    sgtn_destroy(h);
    return SGTN_ERR_ARG;
  }
  int rc = guarded(h, [&] { setup_device(h); });
  if (rc != SGTN_OK) {
    sgtn_destroy(h);
    return rc;
  }
  *out = h;
  return SGTN_OK;
}

int sgtn_set_beta(sgtn_h h, double beta) {
  if (h && !(std::isfinite(beta) && beta >= 0)) {
    h->err = "beta must be finite and >= 0";
    return SGTN_ERR_ARG;
  }
  return guarded(h, [&] { set_beta_device(h, beta); });
}

int sgtn_contract_boundary(sgtn_h h, int32_t chi, int32_t precision, int32_t n_sweeps, double* out_logz,
                           double* out_worst_trunc_sv) {
  return guarded(h, [&] {
    if (!h->beta_set) throw SgtnError(SGTN_ERR_STATE, "set_beta must run first");
    if (chi < 1 || n_sweeps < 0 || n_sweeps > 100) throw SgtnError(SGTN_ERR_ARG, "bad chi or n_sweeps");
    if (precision != SGTN_FP64 && precision != SGTN_FP32 && precision != SGTN_TF32 && precision != SGTN_BF16)
      throw SgtnError(SGTN_ERR_ARG, "precision must be SGTN_FP64, SGTN_FP32, SGTN_TF32 or SGTN_BF16");
    h->precision = precision;
    PrecisionScope ps(h, false);
    contract_boundary(h, chi, n_sweeps);
    if (tc_gemm_take_error(h->st)) throw SgtnError(SGTN_ERR_TIMEOUT, "a tensor-core GEMM timed out");
    if (out_logz) *out_logz = h->logz;
    if (out_worst_trunc_sv) *out_worst_trunc_sv = h->worst_sv;
  });
}

int sgtn_conditionals(sgtn_h h, int32_t step, int32_t count, const int32_t* configs, double* out_p) {
  return guarded(h, [&] {
    PrecisionScope ps(h, true);
    conditionals(h, step, count, configs, out_p);
  });
}

int sgtn_branch_step(sgtn_h h, int32_t step, int32_t M, int32_t in_count, const int32_t* in_configs,
                     const double* in_logp, int32_t* out_configs, double* out_logp, int32_t* out_count,
                     double* io_pd) {
  return guarded(h, [&] {
    PrecisionScope ps(h, true);
    branch_step(h, step, M, in_count, in_configs, in_logp, out_configs, out_logp, out_count, io_pd);
  });
}

int sgtn_search(sgtn_h h, int32_t M, int32_t n_out, int8_t* out_spins, int64_t* out_energy_num, double* out_logp,
                double* out_pd, int32_t* out_count) {
  return guarded(h, [&] {
    PrecisionScope ps(h, true);
    search(h, M, n_out, out_spins, out_energy_num, out_logp, out_pd, out_count);
  });
}

int sgtn_lbp(sgtn_h h, int32_t n_iter, int32_t k, int32_t* out_index, double* out_marginal, int32_t* out_count,
             double* out_change) {
  return guarded(h, [&] {
    if (!h->beta_set) throw SgtnError(SGTN_ERR_STATE, "set_beta must run first");
    if (n_iter < 0 || k < 1 || !out_index || !out_marginal || !out_count)
      throw SgtnError(SGTN_ERR_ARG, "bad n_iter, k or null output");
    for (const auto& S : h->M.sites)
      if (S.d > (1 << 20)) throw SgtnError(SGTN_ERR_ARG, "a site has more than 2^20 states");
    lbp(h, n_iter, k, out_index, out_marginal, out_count, out_change);
  });
}

int sgtn_search_droplets(sgtn_h h, int32_t M, int64_t max_dE_num, int32_t min_hamming, int32_t cap,
                         int8_t* out_spins, int64_t* out_energy_num, double* out_logp, double* out_pd,
                         int32_t* out_ndrop, int64_t* out_dE, int32_t* out_offsets, int32_t* out_flips) {
  return guarded(h, [&] {
    if (cap < 0 || min_hamming < 0 || !out_ndrop || (cap > 0 && (!out_dE || !out_offsets || !out_flips)))
      throw SgtnError(SGTN_ERR_ARG, "bad cap, min_hamming or null output");
    PrecisionScope ps(h, true);
    DropletOpts o;
    o.max_dE = max_dE_num;
    o.min_hamming = min_hamming;
    std::vector<Drop> drops;
    int32_t cnt = 0;
    search(h, M, 1, out_spins, out_energy_num, out_logp, out_pd, &cnt, &o, &drops);
    *out_ndrop = int32_t(drops.size());
    const int nw = std::min<int>(cap, int(drops.size()));
    if (cap > 0) out_offsets[0] = 0;
    for (int i = 0; i < nw; ++i) {
      out_dE[i] = drops[i].dE;
      std::copy(drops[i].flips.begin(), drops[i].flips.end(), out_flips + out_offsets[i]);
      out_offsets[i + 1] = out_offsets[i] + int32_t(drops[i].flips.size());
    }
  });
}

int sgtn_logz_grad(sgtn_h h, double* dJ, double* dh, double* dbeta) {
  return guarded(h, [&] {
    if (!dh || !dbeta || (!dJ && !h->M.ei.empty())) throw SgtnError(SGTN_ERR_ARG, "null output");
    PrecisionScope ps(h, false);
    logz_grad(h, dJ, dh, dbeta);
  });
}

int sgtn_energies(sgtn_h h, int32_t n, const int8_t* spins, int64_t* out) {
  return guarded(h, [&] {
    if (n < 0 || (n > 0 && (!spins || !out))) throw SgtnError(SGTN_ERR_ARG, "bad argument");
    energies(h, n, spins, out);
  });
}

int sgtn_set_search_precision(sgtn_h h, int32_t precision) {
  return guarded(h, [&] {
    if (precision != -1 && precision != SGTN_FP64 && precision != SGTN_FP32 && precision != SGTN_TF32 &&
        precision != SGTN_BF16)
      throw SgtnError(SGTN_ERR_ARG, "search precision must be -1, SGTN_FP64, SGTN_FP32, SGTN_TF32 or SGTN_BF16");
    h->search_precision = precision;
  });
}

int sgtn_set_zipper_window(sgtn_h h, int32_t window) {
  return guarded(h, [&] {
    if (window < 0) throw SgtnError(SGTN_ERR_ARG, "zipper window must be >= 0");
    h->zipper_window = window;
  });
}

int sgtn_set_final_sweeps_fp64(sgtn_h h, int32_t on) {
  return guarded(h, [&] { h->f64_final_sweeps = on != 0; });
}

int sgtn_set_sweep_orthonormalisation(sgtn_h h, int32_t mode) {
  return guarded(h, [&] {
    if (mode != 0 && mode != 1) throw SgtnError(SGTN_ERR_ARG, "sweep orthonormalisation must be 0 (SVD) or 1 (QR)");
    h->sweep_qr = mode == 1;
  });
}

int sgtn_sweep_orthonormalisations(sgtn_h h, int64_t* by_qr, int64_t* by_svd) {
  return guarded(h, [&] {
    if (by_qr) *by_qr = h->sweep_qr_count;
    if (by_svd) *by_svd = h->sweep_svd_count;
  });
}

int sgtn_boundary_info(sgtn_h h, int32_t* unconverged_cuts, int32_t* precision) {
  return guarded(h, [&] {
    if (unconverged_cuts) *unconverged_cuts = h->unconverged_cuts;
    if (precision) *precision = h->precision;
  });
}

int sgtn_site_dims(sgtn_h h, int32_t site, int32_t* d) {
  return guarded(h, [&] {
    if (site < 0 || site >= h->M.R * h->M.C || !d) throw SgtnError(SGTN_ERR_ARG, "bad site");
    *d = h->M.sites[site].d;
  });
}

int sgtn_mps_shape(sgtn_h h, int32_t row, int32_t* phys, int32_t* bond, double* lognorm) {
  return guarded(h, [&] {
    if (!h->boundary_ok) throw SgtnError(SGTN_ERR_STATE, "no boundary MPS");
    if (row < 0 || row >= h->M.R || !phys || !bond) throw SgtnError(SGTN_ERR_ARG, "bad row");
    const MPS& m = h->psi[row];
    for (int c = 0; c < m.C; ++c) phys[c] = m.phys[c];
    for (int c = 0; c <= m.C; ++c) bond[c] = m.bond[c];
    if (lognorm) *lognorm = m.lognorm;
  });
}

int sgtn_mps_tensor(sgtn_h h, int32_t row, int32_t col, double* out) {
  return guarded(h, [&] {
    if (!h->boundary_ok) throw SgtnError(SGTN_ERR_STATE, "no boundary MPS");
    if (row < 0 || row >= h->M.R || col < 0 || col >= h->M.C || !out) throw SgtnError(SGTN_ERR_ARG, "bad index");
    const MPS& m = h->psi[row];
    size_t n = size_t(m.phys[col]) * m.bond[col] * m.bond[col + 1];
    SGTN_CUDA(cudaMemcpyAsync(out, m.t[col], n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    h->sync();
  });
}

void sgtn_stats(int64_t* launches, double* flops, int64_t* evals) {
  if (launches) *launches = g_count.launches;
  if (flops) *flops = g_count.flops;
  if (evals) *evals = g_count.evals;
}

int64_t sgtn_device_allocations(void) { return g_count.device_allocs; }

int sgtn_gemm(int32_t precision, int32_t m, int32_t n, int32_t k, const double* X, const double* Y, double* C,
              void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !X || !Y || !C) return SGTN_ERR_ARG;
  if (precision != SGTN_FP64 && precision != SGTN_FP32 && precision != SGTN_TF32) return SGTN_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  struct Modes {   // the thread's contraction modes for this call only
    Modes(int p) {
      g_compute_f32 = p != SGTN_FP64;
      g_use_tc = p == SGTN_TF32;
    }
    ~Modes() {
      g_compute_f32 = false;
      g_use_tc = false;
    }
  };
  try {
    Modes md(precision);
    gemm(X, false, k, Y, false, n, C, n, m, n, k, 1.0, 0, st);
    if (cudaGetLastError() != cudaSuccess) return SGTN_ERR_CUDA;
    if (precision == SGTN_TF32 && tc_gemm_take_error(st)) return SGTN_ERR_TIMEOUT;
    return SGTN_OK;
  } catch (const SgtnError& e) {
    cudaGetLastError();
    return e.code;
  } catch (const std::exception&) {
    return SGTN_ERR_CUDA;
  }
}

int sgtn_seg_gemm(int32_t precision, int32_t p, int32_t q, int32_t s, int32_t nseg, int32_t nterm, int32_t nx,
                  int32_t ny, const int32_t* seg_ptr, const int32_t* xr, const int32_t* yr, const int32_t* cidx,
                  const double* coef, const double* X, const double* Y, double* O, void* stream) {
  if (p <= 0 || q <= 0 || s <= 0 || nseg <= 0 || nterm < 0 || nx <= 0 || ny <= 0) return SGTN_ERR_ARG;
  if (!seg_ptr || !xr || !yr || !X || !Y || !O || (cidx && !coef)) return SGTN_ERR_ARG;
  if (precision != SGTN_FP64 && precision != SGTN_FP32 && precision != SGTN_TF32 && precision != SGTN_BF16)
    return SGTN_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  struct Modes {   // the thread's contraction modes for this call only
    Modes(int pr) {
      g_compute_f32 = pr != SGTN_FP64;
      g_use_tc = pr == SGTN_TF32 || pr == SGTN_BF16;
      g_tc_bf16 = pr == SGTN_BF16;
    }
    ~Modes() {
      g_compute_f32 = false;
      g_use_tc = false;
      g_tc_bf16 = false;
    }
  };
  try {
    // the term tables are checked on the host before anything is launched:
    // an index out of range would make the kernels read outside X or Y
    {
      std::vector<int32_t> hp(size_t(nseg) + 1), hx(nterm), hy(nterm), hc(cidx ? nterm : 0);
      SGTN_CUDA(cudaMemcpyAsync(hp.data(), seg_ptr, hp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      if (nterm) {
        SGTN_CUDA(cudaMemcpyAsync(hx.data(), xr, hx.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        SGTN_CUDA(cudaMemcpyAsync(hy.data(), yr, hy.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (cidx) SGTN_CUDA(cudaMemcpyAsync(hc.data(), cidx, hc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      }
      SGTN_CUDA(cudaStreamSynchronize(st));
      if (hp[0] != 0 || hp[nseg] != nterm) return SGTN_ERR_ARG;
      for (int g = 0; g < nseg; ++g)
        if (hp[g + 1] < hp[g]) return SGTN_ERR_ARG;
      for (int t = 0; t < nterm; ++t) {
        if (hx[t] < 0 || hx[t] >= nx || hy[t] < 0 || hy[t] >= ny) return SGTN_ERR_ARG;
        if (cidx && (hc[t] < 0 || hc[t] >= nterm)) return SGTN_ERR_ARG;
      }
    }
    Modes md(precision);
    SegGemm a;
    a.name = "seg_gemm";
    a.X = X;
    a.Y = Y;
    a.O = O;
    a.p = p;
    a.q = q;
    a.s = s;
    a.xs_i = q;
    a.xs_k = 1;
    a.xrs = (long long)p * q;
    a.ys_k = s;
    a.ys_j = 1;
    a.yrs = (long long)q * s;
    a.os_i = s;
    a.os_j = 1;
    a.ors = (long long)p * s;
    a.out_by_seg = 1;
    a.seg_ptr = seg_ptr;
    a.xr = xr;
    a.yr = yr;
    a.xc = xr;   // the kernels read a column index per term; with xcs = ycs = 0 it adds nothing
    a.yc = yr;
    a.cidx = cidx;
    a.coef = cidx ? coef : nullptr;
    a.nseg = nseg;
    a.nterm = nterm;
    a.x_rows = (long long)nx * p;
    a.y_rows = (long long)ny * q;
    seg_gemm(a, st);
    if (cudaGetLastError() != cudaSuccess) return SGTN_ERR_CUDA;
    if ((precision == SGTN_TF32 || precision == SGTN_BF16) && tc_gemm_take_error(st)) return SGTN_ERR_TIMEOUT;
    return SGTN_OK;
  } catch (const SgtnError& e) {
    cudaGetLastError();
    return e.code;
  } catch (const std::exception&) {
    return SGTN_ERR_CUDA;
  }
}

int sgtn_cholesky(int32_t n, double shift, const double* G, double* R, double* Rinv, int32_t* status,
                  double* minratio, void* stream) {
  if (n <= 0 || !G || !R || !Rinv || !status) return SGTN_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    g_compute_f32 = false;
    g_use_tc = false;
    cholesky_inv(G, n, shift, R, Rinv, status, st, false, minratio);
    if (cudaGetLastError() != cudaSuccess) return SGTN_ERR_CUDA;
    return SGTN_OK;
  } catch (const SgtnError& e) {
    cudaGetLastError();
    return e.code;
  } catch (const std::exception&) {
    return SGTN_ERR_CUDA;
  }
}

void sgtn_kernel_timing(int32_t enable, int32_t reset) {
  if (reset) ktimer_reset();
  ktimer_enable(enable != 0);
}

int sgtn_kernel_time(const char* name, double* ms, int64_t* launches, double* flops) {
  if (!name || !ms || !launches || !flops) return SGTN_ERR_ARG;
  long long n = 0;
  if (!ktimer_read(name, ms, &n, flops)) return SGTN_ERR_ARG;
  *launches = n;
  return SGTN_OK;
}

int32_t sgtn_kernel_names(char* buf, int32_t cap) {
  const std::string s = ktimer_names();
  if (buf && cap > 0) {
    const size_t n = std::min(s.size(), size_t(cap - 1));
    std::memcpy(buf, s.data(), n);
    buf[n] = '\0';
  }
  return int32_t(s.size());
}

const char* sgtn_last_error(sgtn_h h) { return h ? h->err.c_str() : "null handle"; }

void sgtn_destroy(sgtn_h h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->st);
  if (std::getenv("SGTN_TRACE_MEM")) {
    std::vector<std::pair<size_t, std::string>> v;
    for (auto& kv : h->ws.bufs) v.push_back({kv.second.second, kv.first});
    std::sort(v.rbegin(), v.rend());
    fprintf(stderr, "[sgtn] workspace %.1f MB in %zu buffers:", h->ws.total() / 1048576.0, v.size());
    for (size_t i = 0; i < v.size() && i < 12; ++i) fprintf(stderr, " %s %.1f", v[i].second.c_str(), v[i].first / 1048576.0);
    fprintf(stderr, "\n");
  }
  pool_set_stream(h->st);
  for (auto& m : h->psi) free_mps(m);
  pool_trim(h->st);
  h->ws.release();
  for (void* p : h->allocs) cudaFree(p);
  bool last = false;
  {
    std::lock_guard<std::mutex> lk(g_streams_mu);
    auto it = g_stream_users.find(h->st);
    if (it != g_stream_users.end() && --it->second <= 0) {
      g_stream_users.erase(it);
      last = true;
    }
  }
  if (last) stream_scratch_release(h->st);
  delete h;
}

int sgtn_batch_search(sgtn_h* hs, int32_t n, double beta, int32_t chi, int32_t precision, int32_t n_sweeps,
                      int32_t M, int32_t n_out, int8_t** out_spins, int64_t** out_energy_num, double** out_logp,
                      double* out_logz, double* out_pd, int32_t* out_count, int32_t n_threads, int32_t* status) {
  if (n < 0 || n_threads < 0) return SGTN_ERR_ARG;
  if (n == 0) return SGTN_OK;
  if (!hs || !status || !out_spins || !out_energy_num || !out_logp || !out_logz || !out_pd || !out_count)
    return SGTN_ERR_ARG;
  // handles that share a stream form one group, run in order by one thread
  std::vector<std::vector<int>> groups;
  std::map<cudaStream_t, int> gid;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return SGTN_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return SGTN_ERR_ARG;   // one handle twice would race with itself
    auto it = gid.find(hs[i]->st);
    if (it == gid.end()) {
      gid[hs[i]->st] = int(groups.size());
      groups.push_back({i});
    } else {
      groups[it->second].push_back(i);
    }
  }
  auto run_one = [&](int i) {
    sgtn_h h = hs[i];
    double lz = std::nan("");
    int rc = sgtn_set_beta(h, beta);
    if (rc == SGTN_OK) rc = sgtn_contract_boundary(h, chi, precision, n_sweeps, &lz, nullptr);
    out_logz[i] = lz;
    out_count[i] = 0;
    if (rc == SGTN_OK)
      rc = sgtn_search(h, M, n_out, out_spins[i], out_energy_num[i], out_logp[i], &out_pd[i], &out_count[i]);
    status[i] = rc;
  };
  const int ng = int(groups.size());
  const int nt = std::max(1, n_threads > 0 ? std::min(int(n_threads), ng) : ng);
  std::atomic<int> next{0};
  auto worker = [&] {
    for (int g; (g = next.fetch_add(1)) < ng;)
      for (int i : groups[g]) run_one(i);
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  } catch (const std::exception&) {
    // no more threads: the ones started and this one take the remaining groups
  }
  worker();
  for (auto& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (status[i] != SGTN_OK) return status[i];
  return SGTN_OK;
}

}  // extern "C"
