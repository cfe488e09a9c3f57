// d log Z / dJ_ij, d log Z / dh_i and d log Z / dbeta (paper Eq. 9:
// -beta <s_i s_j>, -beta <s_i>, -<H>) as environment correlators.
//
// For row r the sandwich Z_r = <E_r| T_r |psi_r> joins the bottom-up boundary
// MPS psi_r and an upper boundary MPS E_r of rows 0..r-1, built top-down by the
// same row step (zipper, variational sweeps, cut; Sec. III.B, Fig. 8) applied
// to the transposed row MPOs.  Every Boltzmann factor belongs to exactly one
// row MPO, so each coupling's and field's spin product is averaged in one
// sandwich: with M_c = dZ_r / dW_c (the contraction of everything but column
// c) the average is the sum over the column's terms of M_c * term * s_i s_j,
// divided by Z_r.
//
// Both steps keep the sparse projector form of the columns (Fig. 7):
//  * Column c of T_r reads
//      W[(lam,g)][(lam',g')][u][sigma] = sum_x [Lam x = lam, U x = u] w_x
//        Bv[pd_x][pu sigma] [pul sigma = g] Bh[pr_x][pl lam'] Bdl[pdl lam'][pur sigma] Bdr[pdr_x][g'].
//    Its transpose (out = sigma, in = u) has the same form over the virtual
//    states y = (x, sigma): Lam' y = lam_x nG + pul sigma (no g on the left
//    bond), U' y = sigma, pd' y = u_x with an identity table Bv', pr' y =
//    (pr_x, pur sigma) with Bh'[(pr, pur)][lam'] = Bh[pr][pl lam'] Bdl[pdl lam'][pur]
//    (no e index), pdr' y = pdr_x, and weight w'_y = w_x Bv[pd_x][pu sigma].
//    The top-down pass therefore runs the bottom-up row step unchanged on
//    these columns.
//  * M_c is needed only where some state x reads it: bl = (Lam x, pul sigma),
//    u = U x.  Per distinct (Lam x, U x) pair p and g,
//      N[(p,g)][chl][a'] = sum_a L[a][(lam_p,g)][chl] E[a][u_p][a'],
//    then with AR[(sigma,chl)][(a',br)] = sum_chr A[sigma][chl][chr] R[br][chr][a'],
//      Mp[p][sigma][br] = sum_(chl,a') N[(p, pul sigma)][chl][a'] AR[(sigma,chl)][(a',br)].
//    The weighted terms v(x, sigma, br) = Mp[p_x][sigma][br] * term are
//    reduced to three marginal tables, over (x, sigma), (x, br) and
//    (br, sigma); every spin product of the column depends on one of these
//    pairs, so each correlator is a short sum over one table.  The
//    environments are scaled to unit norm as they are built; each column
//    divides by its own Z_r (the sum of its terms), which the scaling of
//    its environments multiplies alike.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "rowstep.h"

namespace sgtn {

using namespace detail;

namespace {

inline int nblk(long long n) { return int(std::max(1ll, std::min((n + 255) / 256, 148ll * 8))); }

// w'[x nSig + sigma] = w_x Bv[pd_x][pu sigma]
__global__ void tw_kernel(double* tw, const double* w, int d, int nSig, const int32_t* pd_x, const int32_t* s_pu,
                          const double* Bv, int bv_nb) {
  const long long n = (long long)d * nSig;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int x = int(e / nSig), sg = int(e % nSig);
    tw[e] = w[x] * Bv[(long long)pd_x[x] * bv_nb + s_pu[sg]];
  }
}

// Bh'[(pr, pur)][lam'] = Bh[pr][pl lam'] Bdl[pdl lam'][pur]
__global__ void tbh_kernel(double* out, int nPr, int nPur, int nLR, const int32_t* l_pl, const int32_t* l_pdl,
                           const double* Bh, int bh_nb, const double* Bdl, int bdl_nb) {
  const long long n = (long long)nPr * nPur * nLR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int lr = int(e % nLR);
    const long long t = e / nLR;
    const int pur = int(t % nPur), pr = int(t / nPur);
    out[e] = Bh[(long long)pr * bh_nb + l_pl[lr]] * Bdl[(long long)l_pdl[lr] * bdl_nb + pur];
  }
}

// One warp per (x, sigma), lanes over br: v = Mp[p_x][sigma][br] * term,
// summed into Pxs[x][sigma] (warp sum), Pxb[x][br] and Pbs[br][sigma].
__global__ void marginals_kernel(int d, int nSig, int nLR, int nGR, const double* Mp, const int32_t* pair_x,
                                 const double* w, const int32_t* pd_x, const int32_t* pr_x, const int32_t* pdr_x,
                                 const int32_t* s_pu, const int32_t* s_pur, const int32_t* l_pl,
                                 const int32_t* l_pdl, const double* Bv, int bv_nb, const double* Bh, int bh_nb,
                                 const double* Bdl, int bdl_nb, const double* Bdr, int bdr_nb, double* Pxs,
                                 double* Pxb, double* Pbs) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)d * nSig;
  const int nBR = nLR * nGR;
  for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < nw;
       e += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int x = int(e / nSig), sg = int(e % nSig);
    const double wx = w[x] * Bv[(long long)pd_x[x] * bv_nb + s_pu[sg]];
    const double* m = Mp + ((long long)pair_x[x] * nSig + sg) * nBR;
    const long long hr = (long long)pr_x[x] * bh_nb, dr = (long long)pdr_x[x] * bdr_nb;
    const int pur = s_pur[sg];
    double acc = 0.0;
    for (int br = lane; br < nBR; br += 32) {
      const int lr = br / nGR, gr = br % nGR;
      const double v = m[br] * wx * Bh[hr + l_pl[lr]] * Bdl[(long long)l_pdl[lr] * bdl_nb + pur] * Bdr[dr + gr];
      acc += v;
      atomicAdd(&Pxb[(long long)x * nBR + br], v);
      atomicAdd(&Pbs[(long long)br * nSig + sg], v);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Pxs[e] = acc;
  }
}

struct Desc {
  int src_i, bit_i, src_j, bit_j, slot;   // src: 0 none, 1 state x, 2 sigma, 3 lambda', 4 g'
};

__device__ inline double spin_of(int src, int bit, long long st, long long sg, long long lp, long long gp) {
  long long pat = src == 1 ? st : src == 2 ? sg : src == 3 ? lp : gp;
  return src == 0 ? 1.0 : double(1 - 2 * ((pat >> bit) & 1));
}

// One CTA per descriptor: acc[k] = sum over the marginal table that holds both
// of its spins of P * s_i s_j (fixed-order reduction).
__global__ void __launch_bounds__(256) desc_sum_kernel(int d, int nSig, int nLR, int nGR, const double* Pxs,
                                                       const double* Pxb, const double* Pbs, const int64_t* states,
                                                       const int64_t* sig_vals, const int64_t* lam_vals,
                                                       const int64_t* g_vals, const Desc* desc, double* acc) {
  __shared__ double red[8];
  const Desc D = desc[blockIdx.x];
  const int nBR = nLR * nGR;
  // which table: (x, br) if a spin comes from the right bond and the other
  // from x; (br, sigma) for the down-left couplings; (x, sigma) otherwise
  const bool has_b = D.src_i >= 3 || D.src_j >= 3;
  const bool has_x = D.src_i == 1 || D.src_j == 1;
  const int tab = has_b ? (has_x ? 1 : 2) : 0;
  const long long n = tab == 0 ? (long long)d * nSig : tab == 1 ? (long long)d * nBR : (long long)nBR * nSig;
  double s = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    long long stx = 0, sgv = 0, lpv = 0, gpv = 0;
    double P;
    if (tab == 0) {
      const int x = int(e / nSig), sg = int(e % nSig);
      stx = states[x];
      sgv = sig_vals[sg];
      P = Pxs[e];
    } else {
      const int a = int(e / (tab == 1 ? nBR : nSig)), b = int(e % (tab == 1 ? nBR : nSig));
      const int br = tab == 1 ? b : a;
      if (tab == 1) stx = states[a];
      else sgv = sig_vals[b];
      lpv = lam_vals[br / nGR];
      gpv = g_vals[br % nGR];
      P = tab == 1 ? Pxb[e] : Pbs[e];
    }
    s += P * spin_of(D.src_i, D.bit_i, stx, sgv, lpv, gpv) * spin_of(D.src_j, D.bit_j, stx, sgv, lpv, gpv);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    acc[blockIdx.x] = t;
  }
}

// ex[desc[k].slot] = sums[k] / sums[nd]: a column's spin products over its
// own Z_r (the last entry), so the scale of its environments cancels
__global__ void ratio_scatter_kernel(const double* sums, int nd, const Desc* desc, double* ex) {
  for (int k = threadIdx.x; k < nd; k += blockDim.x) ex[desc[k].slot] = sums[k] / sums[nd];
}

// dJ = -beta <ss>, dh = -beta <s>, dbeta = -(sum J <ss> + sum h <s>)
__global__ void finalize_kernel(int nE, int N, const double* ex_all, const int32_t* jn, const int32_t* hn,
                                double denom, double beta, double* dJ, double* dh, double* dbeta) {
  __shared__ double red[32];
  double H = 0;
  for (int i = threadIdx.x; i < nE + N; i += blockDim.x) {
    const double ex = ex_all[i];
    if (i < nE) {
      dJ[i] = -beta * ex;
      H += jn[i] / denom * ex;
    } else {
      dh[i - nE] = -beta * ex;
      H += hn[i - nE] / denom * ex;
    }
  }
  for (int o = 16; o > 0; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = H;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    dbeta[0] = -t;
  }
}

template <class T>
T* to_dev(sgtn_inst* h, const std::vector<T>& v) {
  T* p = nullptr;
  SGTN_CUDA(lib_malloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) SGTN_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->st));
  return p;
}

void free_all(std::vector<double*>& v) {
  for (auto& p : v) dfree(p);
  v.clear();
}

// Bdl of column c: the DL table of (r, c+1), or the unit scalar without a right neighbour
const double* bdl_of(sgtn_inst* h, int r, int c, int& nb) {
  const int C = h->M.C;
  if (c + 1 < C) {
    nb = h->cols[r * C + c].bdl_nb;
    return h->dB[size_t(r * C + c + 1) * 4 + 3];
  }
  double* one = h->ws.get<double>("unit_scalar", 1);
  fill(one, 1, 1.0, h->st);
  nb = 1;
  return one;
}

// The transposed columns of rows 0..R-2 and the correlator index tables
// (host-side tables, uploaded once per handle).
void build_grad_tables(sgtn_inst* h) {
  GradTables& G = h->grad;
  const Model& M = h->M;
  const int R = M.R, C = M.C;
  G.tcols.assign(R * C, Column());
  G.tw.assign(R * C, nullptr);
  G.tbh.assign(R * C, nullptr);
  G.npur.assign(R * C, 1);
  G.xl.assign(R * C, TermTable());
  G.msig.assign(R * C, TermTable());
  G.pair_x.assign(R * C, nullptr);
  G.npairs.assign(R * C, 0);
  G.texp.assign(R * C, 0);
  G.tlexp.assign(R * C, 0);
  auto iota_v = [](int n) {
    std::vector<int32_t> v(n);
    std::iota(v.begin(), v.end(), 0);
    return v;
  };
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) {
      const int rc = r * C + c;
      const HSite& S = M.sites[rc];
      const Column& F = h->cols[rc];
      const HSite* below = M.site(r + 1, c);
      // correlator tables of the forward column
      {
        std::map<std::pair<int32_t, int32_t>, int32_t> pid;
        std::vector<int32_t> px(S.d);
        for (int x = 0; x < S.d; ++x) {
          auto key = std::make_pair(S.Lam.of_state[x], S.U.of_state[x]);
          auto it = pid.find(key);
          if (it == pid.end()) it = pid.emplace(key, int32_t(pid.size())).first;
          px[x] = it->second;
        }
        std::vector<std::pair<int32_t, int32_t>> pairs(pid.size());
        for (auto& kv : pid) pairs[kv.second] = kv.first;
        std::vector<int32_t> xr, yr;
        for (auto& pr : pairs)
          for (int g = 0; g < F.nG; ++g) {
            xr.push_back(pr.first * F.nG + g);   // L block (lam, g)
            yr.push_back(pr.second);             // E block u
          }
        build_pair_table(h, G.xl[rc], xr, yr);
        std::vector<int32_t> sxr(F.nSig, 0);
        if (below)
          for (int sg = 0; sg < F.nSig; ++sg) sxr[sg] = below->U_ul[sg];
        build_pair_table(h, G.msig[rc], sxr, iota_v(F.nSig));
        G.pair_x[rc] = h->upload(px);
        G.npairs[rc] = int(pairs.size());
      }
      if (r + 1 >= R) continue;
      // T_r^T column over y = (x, sigma)
      const int nPur = below->proj[DUR].n;
      G.npur[rc] = nPur;
      Column& K = G.tcols[rc];
      K.r = r;
      K.c = c;
      K.d = S.d * F.nSig;
      K.nLam = F.nLam * F.nG;
      K.nG = 1;
      K.nU = F.nSig;
      K.nSig = F.nU;
      K.nLR = F.nLR;
      K.nGR = F.nGR;
      K.nPd = F.nU;
      K.nPr = F.nPr * nPur;
      K.nPdr = F.nPdr;
      K.nE = 1;
      std::vector<int32_t> lam(K.d), u(K.d), pd(K.d), pr(K.d), pdr(K.d);
      for (int x = 0; x < S.d; ++x)
        for (int sg = 0; sg < F.nSig; ++sg) {
          const int y = x * F.nSig + sg;
          lam[y] = S.Lam.of_state[x] * F.nG + below->U_ul[sg];
          u[y] = sg;
          pd[y] = S.U.of_state[x];
          pr[y] = S.proj[DR_].of_state[x] * nPur + below->U_ur[sg];
          pdr[y] = S.proj[DDR].of_state[x];
        }
      K.lam_x = h->upload(lam);
      K.u_x = h->upload(u);
      K.pd_x = h->upload(pd);
      K.pr_x = h->upload(pr);
      K.pdr_x = h->upload(pdr);
      K.s_pu = h->upload(iota_v(F.nU));
      K.s_pul = K.s_pur = h->upload(std::vector<int32_t>(F.nU, 0));
      K.l_pl = h->upload(iota_v(F.nLR));
      K.l_pdl = h->upload(std::vector<int32_t>(F.nLR, 0));
      K.bv_nb = F.nU;
      K.bh_nb = F.nLR;
      K.bdl_na = K.bdl_nb = 1;
      K.bdr_nb = F.bdr_nb;
      build_column_tables(h, K, lam, u, pd, pr, pdr);
      // Wa' = the identity (Bv' = I, no g, no e): the projected MPS is the MPS
      std::vector<double> eye(size_t(F.nU) * F.nU, 0.0);
      for (int i = 0; i < F.nU; ++i) eye[size_t(i) * F.nU + i] = 1.0;
      K.Wa = h->upload(eye);
      K.Wk = h->dalloc<double>(size_t(K.nK()) * K.nBR());
      G.tw[rc] = h->dalloc<double>(K.d);
      G.tbh[rc] = h->dalloc<double>(size_t(K.nPr) * K.nLR);
    }
  h->sync();
  G.built = true;
}

// Per-beta parts of the transposed columns: w', Bh' and Wk'.
void set_grad_beta(sgtn_inst* h) {
  GradTables& G = h->grad;
  const int R = h->M.R, C = h->M.C;
  for (int r = 0; r + 1 < R; ++r)
    for (int c = 0; c < C; ++c) {
      const int rc = r * C + c;
      const Column& F = h->cols[rc];
      Column& K = G.tcols[rc];
      const double* Bv = h->dB[size_t(rc) * 4 + 1];
      const double* Bh = h->dB[size_t(rc) * 4 + 0];
      const double* Bdr = h->dB[size_t(rc) * 4 + 2];
      int bdl_nb;
      const double* Bdl = bdl_of(h, r, c, bdl_nb);
      tw_kernel<<<nblk(K.d), 256, 0, h->st>>>(G.tw[rc], h->ds[rc].w, F.d, F.nSig, F.pd_x, F.s_pu, Bv, F.bv_nb);
      tbh_kernel<<<nblk((long long)K.nPr * K.nLR), 256, 0, h->st>>>(G.tbh[rc], F.nPr, G.npur[rc], F.nLR, F.l_pl,
                                                                    F.l_pdl, Bh, F.bh_nb, Bdl, bdl_nb);
      build_Wk(K.Wk, K.nPr, 1, K.nPdr, K.nLR, K.nGR, K.l_pl, K.l_pdl, G.tbh[rc], K.bh_nb, Bdr, F.bdr_nb, h->st);
      g_count.launches += 2;
    }
  h->check();
}

// Marginal tables of the weighted terms of column c of row r in the sandwich
// <E_r| T_r |psi_r>; L = left environment [a][bl][chl], Rn = right
// environment [(br, chr)][a'], bra = E_r's tensor [a][u][a'].
void column_marginals(sgtn_inst* h, int r, int c, const double* L, const double* Rn, const Ten& bra, double* Pxs,
                      double* Pxb, double* Pbs) {
  GradTables& G = h->grad;
  cudaStream_t st = h->st;
  const int rc = r * h->M.C + c;
  const Column& K = h->cols[rc];
  const MPS& A = h->psi[r];
  const int nbl = K.nBL(), nbr = K.nBR(), nSig = K.nSig, chl = A.bond[c], chr = A.bond[c + 1];
  const int a = bra.a, ap = bra.b, np = G.npairs[rc];
  const long long Kd = (long long)chl * ap;
  // N[(p, g)][chl][a'] = sum_a L[a][(lam_p, g)][chl] E[a][u_p][a']
  double* N = h->ws.get<double>("gr_N", size_t(G.xl[rc].nseg) * Kd);
  {
    SegGemm n;
    n.name = "grad_env";
    n.X = L;
    n.p = chl;
    n.q = a;
    n.xs_i = 1;
    n.xs_k = (long long)nbl * chl;
    n.xrs = chl;
    n.Y = bra.p;
    n.s = ap;
    n.ys_k = (long long)bra.u * ap;
    n.ys_j = 1;
    n.yrs = ap;
    n.O = N;
    n.os_i = ap;
    n.os_j = 1;
    n.ors = Kd;
    n.out_by_seg = 1;
    n.seg_ptr = G.xl[rc].seg_ptr;
    n.xr = G.xl[rc].xr;
    n.xc = G.xl[rc].xc;
    n.yr = G.xl[rc].yr;
    n.yc = G.xl[rc].yc;
    n.nseg = G.xl[rc].nseg;
    n.nterm = G.xl[rc].nterm;
    seg_gemm(n, st);
  }
  // AR[(sigma, chl)][(a', br)] = sum_chr A[sigma][chl][chr] R[br][chr][a']
  double* Rp = h->ws.get<double>("gr_Rp", size_t(chr) * ap * nbr);
  {
    int dims[3] = {nbr, chr, ap}, perm[3] = {1, 2, 0};
    permute_nd(Rn, 3, dims, perm, Rp, st);
  }
  double* AR = h->ws.get<double>("gr_AR", size_t(nSig) * Kd * nbr);
  gemm(A.t[c], false, chr, Rp, false, (long long)ap * nbr, AR, (long long)ap * nbr, nSig * chl, ap * nbr, chr, 1.0, 0,
       st);
  // Mp[p][sigma][br] = sum_(chl, a') N[(p, pul sigma)][(chl, a')] AR[sigma][(chl, a')][br]
  double* Mp = h->ws.get<double>("gr_Mp", size_t(np) * nSig * nbr);
  {
    SegGemm m;
    m.name = "grad_env";
    m.X = N;
    m.p = np;
    m.q = int(Kd);
    m.xs_i = (long long)K.nG * Kd;
    m.xs_k = 1;
    m.xrs = Kd;
    m.Y = AR;
    m.s = nbr;
    m.ys_k = nbr;
    m.ys_j = 1;
    m.yrs = Kd * nbr;
    m.O = Mp;
    m.os_i = (long long)nSig * nbr;
    m.os_j = 1;
    m.ors = nbr;
    m.out_by_seg = 1;
    m.seg_ptr = G.msig[rc].seg_ptr;
    m.xr = G.msig[rc].xr;
    m.xc = G.msig[rc].xc;
    m.yr = G.msig[rc].yr;
    m.yc = G.msig[rc].yc;
    m.nseg = G.msig[rc].nseg;
    m.nterm = G.msig[rc].nterm;
    seg_gemm(m, st);
  }
  SGTN_CUDA(cudaMemsetAsync(Pxb, 0, size_t(K.d) * nbr * sizeof(double), st));
  SGTN_CUDA(cudaMemsetAsync(Pbs, 0, size_t(nbr) * nSig * sizeof(double), st));
  int bdl_nb;
  const double* Bdl = bdl_of(h, r, c, bdl_nb);
  const long long warps = (long long)K.d * nSig;
  marginals_kernel<<<int(std::max(1ll, std::min((warps + 7) / 8, 148ll * 16))), 256, 0, st>>>(
      K.d, nSig, K.nLR, K.nGR, Mp, G.pair_x[rc], h->ds[rc].w, K.pd_x, K.pr_x, K.pdr_x, K.s_pu, K.s_pur, K.l_pl,
      K.l_pdl, h->dB[size_t(rc) * 4 + 1], K.bv_nb, h->dB[size_t(rc) * 4 + 0], K.bh_nb, Bdl, bdl_nb,
      h->dB[size_t(rc) * 4 + 2], K.bdr_nb, Pxs, Pxb, Pbs);
  ++g_count.launches;
}

}  // namespace

void logz_grad(sgtn_inst* h, double* dJ, double* dh, double* dbeta) {
  if (!h->boundary_ok) throw SgtnError(-2, "contract_boundary must run first");
  if (h->n_sweeps < 1) throw SgtnError(-1, "gradients need n_sweeps >= 1 in contract_boundary");
  const int R = h->M.R, C = h->M.C, N = h->M.N;
  const int nE = int(h->M.ei.size());
  cudaStream_t st = h->st;
  if (!h->grad.built) build_grad_tables(h);
  set_grad_beta(h);
  GradTables& G = h->grad;
  std::fill(G.texp.begin(), G.texp.end(), 0);
  std::fill(G.tlexp.begin(), G.tlexp.end(), 0);
  // top-down upper boundary MPSs E_0..E_{R-1}: E_{r+1} ~ T_r^T E_r
  std::vector<MPS> E(R);
  E[0].C = C;
  E[0].phys.assign(C, 1);
  E[0].bond.assign(C + 1, 1);
  E[0].t.assign(C, nullptr);
  for (int c = 0; c < C; ++c) {
    E[0].t[c] = dmalloc(1);
    fill(E[0].t[c], 1, 1.0, st);
  }
  E[0].valid = true;
  double worst = 0;
  for (int r = 0; r + 1 < R; ++r) {
    RowCtx X;
    X.h = h;
    X.r = r;
    X.cols = &G.tcols[r * C];
    X.w = &G.tw[r * C];
    X.sexp = &G.texp[size_t(r) * C];
    X.lexp = &G.tlexp[size_t(r) * C];
    row_step_ctx(X, E[r], h->chi, h->n_sweeps, E[r + 1], worst);
  }
  // expectations: slots [edges | spins]
  double* acc = dmalloc(nE + N);
  SGTN_CUDA(cudaMemsetAsync(acc, 0, (nE + N) * sizeof(double), st));
  // descriptors per (row, column)
  std::vector<std::vector<Desc>> desc(R * C);
  auto local_bit = [&](const HSite& S, int spin) {
    return int(std::find(S.spins.begin(), S.spins.end(), spin) - S.spins.begin());
  };
  auto pos = [](const std::vector<int>& bits, int b) { return int(std::find(bits.begin(), bits.end(), b) - bits.begin()); };
  for (int e = 0; e < nE; ++e) {
    int i = h->M.ei[e], j = h->M.ej[e];
    int si = h->M.site_of_spin[i], sj = h->M.site_of_spin[j];
    int ri = si / C, ci = si % C, rj = sj / C, cj = sj % C;
    if (ri > rj || (ri == rj && ci > cj)) {
      std::swap(i, j);
      std::swap(si, sj);
      std::swap(ri, rj);
      std::swap(ci, cj);
    }
    const HSite& S = h->M.sites[si];
    Desc D{0, 0, 0, 0, e};
    int owner_r = ri, owner_c = ci;
    if (si == sj) {
      D = {1, local_bit(S, i), 1, local_bit(S, j), e};
    } else if (rj == ri && cj == ci + 1) {          // horizontal: j from lambda' of (r, c+1)
      const HSite& T = h->M.sites[sj];
      D = {1, local_bit(S, i), 3, pos(T.Lam.bits, local_bit(T, j)), e};
    } else if (rj == ri + 1 && cj == ci) {          // vertical: j from sigma of (r+1, c)
      const HSite& T = h->M.sites[sj];
      D = {1, local_bit(S, i), 2, pos(T.U.bits, local_bit(T, j)), e};
    } else if (rj == ri + 1 && cj == ci + 1) {      // down-right: j from g' of (r+1, c+1)
      const HSite& T = h->M.sites[sj];
      D = {1, local_bit(S, i), 4, pos(T.proj[DUL].bits, local_bit(T, j)), e};
    } else if (rj == ri + 1 && cj == ci - 1) {      // down-left: owned by column c-1 = cj
      const HSite& T = h->M.sites[sj];
      D = {3, pos(S.Lam.bits, local_bit(S, i)), 2, pos(T.U.bits, local_bit(T, j)), e};
      owner_c = cj;
    } else {
      throw SgtnError(-1, "edge between non-neighbouring clusters");
    }
    desc[owner_r * C + owner_c].push_back(D);
  }
  for (int s = 0; s < R * C; ++s) {
    const HSite& S = h->M.sites[s];
    for (size_t j = 0; j < S.spins.size(); ++j) {
      desc[s].push_back({1, int(j), 0, 0, nE + S.spins[j]});
    }
  }
  // per-row sandwich
  for (int r = 0; r < R; ++r) {
    RowCtx X;
    X.h = h;
    X.r = r;
    X.A = &h->psi[r];
    X.sexp = &h->theta_exp[size_t(r) * C];   // the bottom-up pass's exponents (any scale cancels here)
    X.lexp = &h->lenv_exp[size_t(r) * C];
    compute_ahat(X);
    // bra tensors of E_r as [a][u][b]
    std::vector<Ten> bra(C);
    for (int c = 0; c < C; ++c) {
      bra[c].a = E[r].bond[c];
      bra[c].u = E[r].phys[c];
      bra[c].b = E[r].bond[c + 1];
      bra[c].p = dmalloc(bra[c].n());
      permute3(E[r].t[c], bra[c].u, bra[c].a, bra[c].b, bra[c].p, st);
    }
    std::vector<double*> Re(C, nullptr), Le(C, nullptr);
    Re[C - 1] = dmalloc(1);
    fill(Re[C - 1], 1, 1.0, st);
    // environments scaled to unit norm as they are built (their raw size
    // follows the Boltzmann factors and can leave the floating-point range)
    // (mixed arithmetic: a step's weight exponent is adapted when the
    // result's norm leaves 2^+-100, as in the row step)
    double scale = 0.0;
    for (int c = C - 1; c > 0; --c) {
      const long long n = (long long)X.col(c).nBL() * X.chl(c) * bra[c].a;
      for (int tries = 0;; ++tries) {
        double* Th = theta_of(X, c, Re[c], bra[c].b);
        double* Rn = update_R(X, c, Th, bra[c]);
        const int step = (g_compute_f32 && tries < 4) ? exp_step(norm_value(h, Rn, n)) : 0;
        if (step == 0) {
          Re[c - 1] = Rn;
          break;
        }
        X.sexp[c] += step;
        dfree(Rn);
      }
      normalise(h, Re[c - 1], n, scale);
    }
    Le[0] = dmalloc(1);
    fill(Le[0], 1, 1.0, st);
    for (int c = 0; c + 1 < C; ++c) Le[c + 1] = update_L_adapt(X, c, Le[c], bra[c]);
    for (int c = 0; c < C; ++c) {
      const int rc = r * C + c;
      const Column& K = X.col(c);
      const int nbr = K.nBR(), nSig = K.nSig;
      double* Pxs = dmalloc((long long)K.d * nSig);
      double* Pxb = dmalloc((long long)K.d * nbr);
      double* Pbs = dmalloc((long long)nbr * nSig);
      column_marginals(h, r, c, Le[c], Re[c], bra[c], Pxs, Pxb, Pbs);
      // descriptors of this column, then its Z_r
      std::vector<Desc> dv = desc[rc];
      const int nd = int(dv.size());
      dv.push_back({0, 0, 0, 0, -1});
      if (nd > 0) {
        const HSite& S = h->M.sites[rc];
        const HSite* below = h->M.site(r + 1, c);
        const HSite* right = h->M.site(r, c + 1);
        const HSite* br_ = h->M.site(r + 1, c + 1);
        std::vector<int64_t> zero1(1, 0);
        int64_t* st_d = to_dev(h, S.states);
        int64_t* sg_d = to_dev(h, below ? below->U.vals : zero1);
        int64_t* lp_d = to_dev(h, right ? right->Lam.vals : zero1);
        int64_t* gp_d = to_dev(h, br_ ? br_->proj[DUL].vals : zero1);
        Desc* dd = to_dev(h, dv);
        double* accz = dmalloc(int(dv.size()));
        desc_sum_kernel<<<int(dv.size()), 256, 0, st>>>(K.d, nSig, K.nLR, K.nGR, Pxs, Pxb, Pbs, st_d, sg_d, lp_d,
                                                        gp_d, dd, accz);
        ++g_count.launches;
        ratio_scatter_kernel<<<1, 256, 0, st>>>(accz, nd, dd, acc);
        ++g_count.launches;
        h->sync();
        cudaFree(dd);
        cudaFree(st_d);
        cudaFree(sg_d);
        cudaFree(lp_d);
        cudaFree(gp_d);
        dfree(accz);
      }
      dfree(Pxs);
      dfree(Pxb);
      dfree(Pbs);
    }
    for (auto& t : bra) dfree(t.p);
    for (double*& p : X.Ahat) dfree(p);
    free_all(Re);
    free_all(Le);
  }
  // outputs
  double *ddJ = dmalloc(std::max(nE, 1)), *ddh = dmalloc(N), *ddb = dmalloc(1);
  int32_t* jn = to_dev(h, h->M.jn.empty() ? std::vector<int32_t>(1, 0) : h->M.jn);
  int32_t* hn = to_dev(h, h->M.hn);
  finalize_kernel<<<1, 1024, 0, st>>>(nE, N, acc, jn, hn, double(h->M.denom), h->beta, ddJ, ddh, ddb);
  ++g_count.launches;
  h->check();
  if (nE) SGTN_CUDA(cudaMemcpyAsync(dJ, ddJ, nE * sizeof(double), cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(dh, ddh, N * sizeof(double), cudaMemcpyDeviceToHost, st));
  SGTN_CUDA(cudaMemcpyAsync(dbeta, ddb, sizeof(double), cudaMemcpyDeviceToHost, st));
  h->sync();
  dfree(ddJ);
  dfree(ddh);
  dfree(ddb);
  dfree(acc);
  cudaFree(jn);
  cudaFree(hn);
  for (auto& m : E) free_mps(m);
}

}  // namespace sgtn
