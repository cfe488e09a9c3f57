// Loopy belief propagation over the clusters of the Potts model (paper
// Sec. IV): approximate marginals of every cluster's states, used to keep the
// most probable states of each cluster before the tensor-network contraction
// (the local dimensional reduction).
//
// Messages are indexed by the projected classes of Eq. (4).  For a site s and
// a neighbour t (any site that shares a coupling with s):
//   mu_{s->t}(a) = sum_{x: P^{st}(x) = a} w_x prod_{t' != t} nu_{t'->s}(P^{st'}(x))
//   nu_{s->t}(b) = sum_a exp(-beta Ebar^{st}[a, b]) mu_{s->t}(a)
//   p(x_s)      ~ w_x prod_t nu_{t->s}(P^{st}(x))
// with w_x = exp(-beta (E_x - E_min)) and the bond factors of set_beta.
// Schedule: synchronous (all mu from the previous nu, then all nu), nu starts
// at one and is scaled to sum 1 after every update; the reported change is
// the largest |nu_new - nu_old| of the last iteration.
//
// Layout: one "edge" per ordered neighbour pair (s, direction); the incoming
// message nu_{t->s} and the outgoing mu_{s->t} of an edge share its offset in
// two pools (indexed by the classes of s toward t).  Every reduction is a
// fixed-order warp or block sum: results do not depend on scheduling.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <vector>

#include "handle.h"

namespace sgtn {

namespace {

struct LbpEdge {
  int s = 0, t = 0, dd = 0, na = 1, partner = -1;
  long long off = 0;                    // offset of this edge's messages in the pools
  const double* B = nullptr;            // bond factor exp(-beta (Ebar - min))
  long long sa = 0, sb = 0;             // B(a, b) = B[a sa + b sb], a: class of s, b: class of t
  const int32_t* cls = nullptr;         // class of each state of s toward t
  const int32_t* csr_ptr = nullptr;     // states of s grouped by class toward t
  const int32_t* csr_idx = nullptr;
};

__device__ __forceinline__ double lbp_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (blockDim.x a multiple of 32, at most 1024).
__device__ double lbp_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = lbp_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// mu_{s->t}(a) for every (edge, class) item: one warp per item
__global__ void lbp_mu_kernel(const LbpEdge* E, const int32_t* site_ptr, const int32_t* site_edges,
                              const double* const* w, const double* nu, double* mu, const int32_t* item_e,
                              const int32_t* item_a, int nitems) {
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= nitems) return;
  const int e = item_e[item], a = item_a[item];
  const LbpEdge& ed = E[e];
  const int s = ed.s;
  const int e0 = site_ptr[s], e1 = site_ptr[s + 1];
  const double* ws = w[s];
  double acc = 0.0;
  for (int p = ed.csr_ptr[a] + lane; p < ed.csr_ptr[a + 1]; p += 32) {
    const int x = ed.csr_idx[p];
    double v = ws[x];
    for (int q = e0; q < e1; ++q) {
      const int e2 = site_edges[q];
      if (e2 == e) continue;
      v *= nu[E[e2].off + E[e2].cls[x]];
    }
    acc += v;
  }
  acc = lbp_warp_sum(acc);
  if (lane == 0) mu[ed.off + a] = acc;
}

// nu_{s->t} = B^T mu_{s->t} (unscaled) into the partner edge's slot.  Grid
// (edge, chunk of 64 b).  B is read along its contiguous index: with
// B(a, b) = B[a sa + b sb], sb == 1 puts consecutive b in consecutive threads
// (one thread per b, loop over a); sa == 1 gives one warp per b whose lanes
// run over a.
__global__ void lbp_nu_kernel(const LbpEdge* E, const double* mu, double* nu_new) {
  const LbpEdge& ed = E[blockIdx.x];
  const LbpEdge& pt = E[ed.partner];
  const int nb = pt.na, b0 = blockIdx.y * 64;
  if (b0 >= nb) return;
  const double* m = mu + ed.off;
  if (ed.sb == 1) {
    const int b = b0 + threadIdx.x;
    if (threadIdx.x < 64 && b < nb) {
      double v = 0.0;
      for (int a = 0; a < ed.na; ++a) v = fma(ed.B[a * ed.sa + b], m[a], v);
      nu_new[pt.off + b] = v;
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = b0 + warp; b < min(nb, b0 + 64); b += nw) {
      const double* Bb = ed.B + (long long)b * ed.sb;
      double v = 0.0;
      for (int a = lane; a < ed.na; a += 32) v = fma(Bb[a], m[a], v);
      v = lbp_warp_sum(v);
      if (lane == 0) nu_new[pt.off + b] = v;
    }
  }
}

// scale every new message to sum 1; chg[e] = largest change against the
// previous one (one CTA per edge, the message indexed like edge e's partner)
__global__ void lbp_norm_kernel(const LbpEdge* E, const double* nu_old, double* nu_new, double* chg) {
  __shared__ double red[32];
  const LbpEdge& pt = E[E[blockIdx.x].partner];
  const int nb = pt.na;
  double part = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) part += nu_new[pt.off + b];
  const double tot = lbp_block_sum(part, red);
  double mx = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double v = nu_new[pt.off + b] / tot;
    nu_new[pt.off + b] = v;
    mx = fmax(mx, fabs(v - nu_old[pt.off + b]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    chg[blockIdx.x] = mm;
  }
}

// marginals of one site per CTA, scaled to sum 1
__global__ void lbp_marginal_kernel(const LbpEdge* E, const int32_t* site_ptr, const int32_t* site_edges,
                                    const double* const* w, const int32_t* dsite, const long long* moff,
                                    const double* nu, double* marg) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const int d = dsite[s], e0 = site_ptr[s], e1 = site_ptr[s + 1];
  double* out = marg + moff[s];
  double part = 0.0;
  for (int x = threadIdx.x; x < d; x += blockDim.x) {
    double v = w[s][x];
    for (int q = e0; q < e1; ++q) {
      const int e = site_edges[q];
      v *= nu[E[e].off + E[e].cls[x]];
    }
    out[x] = v;
    part += v;
  }
  const double tot = lbp_block_sum(part, red);
  for (int x = threadIdx.x; x < d; x += blockDim.x) out[x] /= tot;
}

// rank of every state of a site (larger marginal first, ties to the smaller
// index) and the k first written out; one CTA per site, marginals staged in
// shared memory when they fit.  Marginals are non-negative, so their bit
// patterns order like their values: the comparisons run on the integer pipe
// (B300 issues FP64 comparisons at its low FP64 rate).
__global__ void lbp_rank_kernel(const int32_t* dsite, const long long* moff, const double* marg, int k,
                                int32_t* out_idx, double* out_p, int smem_cap) {
  extern __shared__ long long sk[];
  const int s = blockIdx.x, d = dsite[s];
  const double* m = marg + moff[s];
  const long long* mk = reinterpret_cast<const long long*>(m);
  const bool staged = d <= smem_cap;
  if (staged)
    for (int x = threadIdx.x; x < d; x += blockDim.x) sk[x] = __double_as_longlong(m[x]);
  __syncthreads();
  const long long* b = staged ? sk : mk;
  for (int x = threadIdx.x; x < d; x += blockDim.x) {
    const long long bx = b[x];
    int rank = 0;
    for (int y = 0; y < d; ++y) {
      const long long by = b[y];
      rank += (by > bx) | ((by == bx) & (y < x));
    }
    if (rank < k) {
      out_idx[(long long)s * k + rank] = x;
      out_p[(long long)s * k + rank] = __longlong_as_double(bx);
    }
  }
}

}  // namespace

void lbp(sgtn_inst* h, int n_iter, int k, int32_t* out_index, double* out_marginal, int32_t* out_count,
         double* out_change) {
  const Model& M = h->M;
  const int R = M.R, C = M.C, ns = R * C;
  cudaStream_t st = h->st;
  // edges: ordered neighbour pairs that share a coupling
  std::vector<LbpEdge> E;
  std::vector<int32_t> site_ptr(ns + 1, 0), site_edges;
  std::vector<std::vector<int32_t>> csr_ptr_h, csr_idx_h;
  std::vector<int> edge_of(size_t(ns) * 8, -1);
  long long off = 0;
  for (int s = 0; s < ns; ++s) {
    const HSite& S = M.sites[s];
    site_ptr[s] = int32_t(site_edges.size());
    for (int dd = 0; dd < 8; ++dd) {
      const HSite* T = M.site(S.r + kDr[dd], S.c + kDc[dd]);
      if (!T || S.coupled[dd].empty()) continue;
      LbpEdge ed;
      ed.s = s;
      ed.t = T->r * C + T->c;
      ed.dd = dd;
      ed.na = S.proj[dd].n;
      ed.off = off;
      off += ed.na;
      const int slot = Model::tab_slot(Dir(dd));
      if (slot >= 0) {
        ed.B = h->dB[size_t(s) * 4 + slot];
        ed.sa = M.tab[size_t(s) * 4 + slot].nB;
        ed.sb = 1;
      } else {
        ed.B = h->dB[size_t(ed.t) * 4 + Model::tab_slot(Dir(kOpp[dd]))];
        ed.sa = 1;
        ed.sb = ed.na;
      }
      ed.cls = h->ds[s].cls[dd];
      // states grouped by class (stable: increasing state index within a class)
      std::vector<int32_t> ptr(ed.na + 1, 0), idx(S.d);
      for (int x = 0; x < S.d; ++x) ++ptr[S.proj[dd].of_state[x] + 1];
      for (int a = 0; a < ed.na; ++a) ptr[a + 1] += ptr[a];
      std::vector<int32_t> fillp(ptr.begin(), ptr.end() - 1);
      for (int x = 0; x < S.d; ++x) idx[fillp[S.proj[dd].of_state[x]]++] = x;
      csr_ptr_h.push_back(std::move(ptr));
      csr_idx_h.push_back(std::move(idx));
      edge_of[size_t(s) * 8 + dd] = int(E.size());
      site_edges.push_back(int32_t(E.size()));
      E.push_back(ed);
    }
  }
  site_ptr[ns] = int32_t(site_edges.size());
  const int ne = int(E.size());
  for (auto& ed : E) {
    ed.partner = edge_of[size_t(ed.t) * 8 + kOpp[ed.dd]];
    if (ed.partner < 0) throw SgtnError(-2, "inconsistent coupling structure");
  }
  // device copies (temporary, released at the end of the call)
  std::vector<void*> tmp;
  auto up = [&](const void* src, size_t bytes) {
    void* p = pool_alloc(std::max<size_t>(bytes, 8));
    if (bytes) SGTN_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st));
    tmp.push_back(p);
    return p;
  };
  for (int e = 0; e < ne; ++e) {
    E[e].csr_ptr = static_cast<const int32_t*>(up(csr_ptr_h[e].data(), csr_ptr_h[e].size() * 4));
    E[e].csr_idx = static_cast<const int32_t*>(up(csr_idx_h[e].data(), csr_idx_h[e].size() * 4));
  }
  std::vector<int32_t> item_e, item_a;
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < E[e].na; ++a) item_e.push_back(e), item_a.push_back(a);
  std::vector<const double*> wp(ns);
  std::vector<int32_t> dsite(ns);
  std::vector<long long> moff(ns + 1, 0);
  int dmax = 1;
  for (int s = 0; s < ns; ++s) {
    wp[s] = h->ds[s].w;
    dsite[s] = M.sites[s].d;
    moff[s + 1] = moff[s] + M.sites[s].d;
    dmax = std::max(dmax, M.sites[s].d);
  }
  auto* dE = static_cast<LbpEdge*>(up(E.data(), E.size() * sizeof(LbpEdge)));
  auto* dsp = static_cast<int32_t*>(up(site_ptr.data(), site_ptr.size() * 4));
  auto* dse = static_cast<int32_t*>(up(site_edges.data(), site_edges.size() * 4));
  auto* die = static_cast<int32_t*>(up(item_e.data(), item_e.size() * 4));
  auto* dia = static_cast<int32_t*>(up(item_a.data(), item_a.size() * 4));
  auto* dw = static_cast<const double* const*>(up(wp.data(), wp.size() * sizeof(double*)));
  auto* dds = static_cast<int32_t*>(up(dsite.data(), dsite.size() * 4));
  auto* dmo = static_cast<long long*>(up(moff.data(), moff.size() * 8));
  const size_t nmsg = size_t(std::max<long long>(off, 1));
  double* nu = static_cast<double*>(pool_alloc(nmsg * 8));
  double* nu2 = static_cast<double*>(pool_alloc(nmsg * 8));
  double* mu = static_cast<double*>(pool_alloc(nmsg * 8));
  double* chg = static_cast<double*>(pool_alloc(std::max(ne, 1) * 8));
  double* marg = static_cast<double*>(pool_alloc(size_t(std::max<long long>(moff[ns], 1)) * 8));
  int32_t* oidx = static_cast<int32_t*>(pool_alloc(std::max<size_t>(size_t(ns) * k * 4, 8)));
  double* op = static_cast<double*>(pool_alloc(std::max<size_t>(size_t(ns) * k * 8, 8)));
  for (void* p : {(void*)nu, (void*)nu2, (void*)mu, (void*)chg, (void*)marg, (void*)oidx, (void*)op}) tmp.push_back(p);
  fill(nu, (long long)nmsg, 1.0, st);
  SGTN_CUDA(cudaMemsetAsync(chg, 0, std::max(ne, 1) * 8, st));
  const int nitems = int(item_e.size());
  int max_na = 1;
  for (const auto& ed : E) max_na = std::max(max_na, ed.na);
  for (int it = 0; it < n_iter && ne > 0; ++it) {
    {
      KTimer kt("lbp_mu", st);
      lbp_mu_kernel<<<(nitems + 7) / 8, 256, 0, st>>>(dE, dsp, dse, dw, nu, mu, die, dia, nitems);
    }
    {
      KTimer kt("lbp_nu", st);
      lbp_nu_kernel<<<dim3(ne, (max_na + 63) / 64), 256, 0, st>>>(dE, mu, nu2);
      lbp_norm_kernel<<<ne, 256, 0, st>>>(dE, nu, nu2, chg);
    }
    g_count.launches += 3;
    std::swap(nu, nu2);
  }
  {
    KTimer kt("lbp_marginal", st);
    lbp_marginal_kernel<<<ns, 256, 0, st>>>(dE, dsp, dse, dw, dds, dmo, nu, marg);
  }
  const int smem_cap = 200 * 1024 / 8;
  static const bool attr = [] {
    cudaFuncSetAttribute(lbp_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  SGTN_CUDA(cudaMemsetAsync(oidx, 0xff, size_t(ns) * k * 4, st));
  {
    KTimer kt("lbp_rank", st);
    lbp_rank_kernel<<<ns, 1024, size_t(std::min(dmax, smem_cap)) * 8, st>>>(dds, dmo, marg, k, oidx, op, smem_cap);
  }
  g_count.launches += 2;
  h->check();
  std::vector<double> hchg(std::max(ne, 1), 0.0);
  SGTN_CUDA(cudaMemcpyAsync(out_index, oidx, size_t(ns) * k * 4, cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(out_marginal, op, size_t(ns) * k * 8, cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(hchg.data(), chg, hchg.size() * 8, cudaMemcpyDeviceToHost, st));
  h->sync();
  for (int s = 0; s < ns; ++s) out_count[s] = std::min(k, M.sites[s].d);
  if (out_change) *out_change = n_iter > 0 ? *std::max_element(hchg.begin(), hchg.end()) : 0.0;
  for (void* p : tmp) pool_free(p);
}

}  // namespace sgtn
