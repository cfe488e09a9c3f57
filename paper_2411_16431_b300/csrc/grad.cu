// d log Z / dJ_ij, d log Z / dh_i and d log Z / dbeta (paper Eq. 9:
// -beta <s_i s_j>, -beta <s_i>, -<H>) as environment correlators.
//
// For row r the sandwich Z_r = <E_r| T_r |psi_r> joins the bottom-up boundary
// MPS psi_r and an upper boundary MPS E_r of rows 0..r-1, built top-down by the
// same row step (zipper, variational sweeps, cut) applied to the transposed
// row MPOs.  Every Boltzmann factor belongs to exactly one row MPO, so each
// coupling's and field's spin product is averaged in one sandwich: with
// M_c = dZ_r / dW_c (the contraction of everything but column c) the average
// is sum over the column's per-state terms of M_c * term * s_i s_j / Z_r.
// The row MPOs are handled as dense column tensors here, which bounds this
// path to instances whose column tensors nBL x nBR x nU x nSig are small.
#include <algorithm>
#include <cmath>

#include "rowstep.h"

namespace sgtn {

using namespace detail;

namespace {

// W[bl][br][u][sigma] = sum_x [Lam x, U x] w_x Bv Bh Bdl Bdr  (definition of the MPO column)
__global__ void densify_kernel(double* W, int d, int nG, int nU, int nSig, int nLR, int nGR, const double* w,
                               const int32_t* lam_x, const int32_t* u_x, const int32_t* pd_x, const int32_t* pr_x,
                               const int32_t* pdr_x, const int32_t* s_pu, const int32_t* s_pul, const int32_t* s_pur,
                               const int32_t* l_pl, const int32_t* l_pdl, const double* Bv, int bv_nb,
                               const double* Bh, int bh_nb, const double* Bdl, int bdl_nb, const double* Bdr,
                               int bdr_nb, long long n) {
  const long long nBR = (long long)nLR * nGR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int sg = int(e % nSig);
    long long t = e / nSig;
    int u = int(t % nU);
    t /= nU;
    long long br = t % nBR;
    long long bl = t / nBR;
    int lam = int(bl / nG), g = int(bl % nG);
    double acc = 0.0;
    if (s_pul[sg] == g) {
      int lamR = int(br / nGR), gR = int(br % nGR);
      for (int x = 0; x < d; ++x) {
        if (lam_x[x] != lam || u_x[x] != u) continue;
        acc += w[x] * Bv[(long long)pd_x[x] * bv_nb + s_pu[sg]] * Bh[(long long)pr_x[x] * bh_nb + l_pl[lamR]] *
               Bdl[(long long)l_pdl[lamR] * bdl_nb + s_pur[sg]] * Bdr[(long long)pdr_x[x] * bdr_nb + gR];
      }
    }
    W[e] = acc;
  }
}

struct Desc {
  int src_i, bit_i, src_j, bit_j, slot;   // src: 0 none, 1 state x, 2 sigma, 3 lambda', 4 g'
};

__device__ inline double spin_of(int src, int bit, long long st, long long sg, long long lp, long long gp) {
  long long pat = src == 1 ? st : src == 2 ? sg : src == 3 ? lp : gp;
  return src == 0 ? 1.0 : double(1 - 2 * ((pat >> bit) & 1));
}

// acc[desc.slot] += sum over (x, sigma, lambda', g') of M * term * s_i s_j
__global__ void edge_sum_kernel(int d, int nG, int nU, int nSig, int nLR, int nGR, const double* M, const double* w,
                                const int32_t* lam_x, const int32_t* u_x, const int32_t* pd_x, const int32_t* pr_x,
                                const int32_t* pdr_x, const int32_t* s_pu, const int32_t* s_pul, const int32_t* s_pur,
                                const int32_t* l_pl, const int32_t* l_pdl, const double* Bv, int bv_nb,
                                const double* Bh, int bh_nb, const double* Bdl, int bdl_nb, const double* Bdr,
                                int bdr_nb, const int64_t* states, const int64_t* sig_vals, const int64_t* lam_vals,
                                const int64_t* g_vals, int ndesc, const Desc* desc, double* acc) {
  extern __shared__ double part[];   // ndesc
  for (int i = threadIdx.x; i < ndesc; i += blockDim.x) part[i] = 0.0;
  __syncthreads();
  const long long nBR = (long long)nLR * nGR;
  const long long n = (long long)d * nSig * nBR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int sg = int(e % nSig);
    long long t = e / nSig;
    long long br = t % nBR;
    int x = int(t / nBR);
    int lamR = int(br / nGR), gR = int(br % nGR);
    double term = w[x] * Bv[(long long)pd_x[x] * bv_nb + s_pu[sg]] * Bh[(long long)pr_x[x] * bh_nb + l_pl[lamR]] *
                  Bdl[(long long)l_pdl[lamR] * bdl_nb + s_pur[sg]] * Bdr[(long long)pdr_x[x] * bdr_nb + gR];
    long long bl = (long long)lam_x[x] * nG + s_pul[sg];
    double m = M[((bl * nU + u_x[x]) * nBR + br) * nSig + sg];
    double v = m * term;
    if (v == 0.0) continue;
    long long stx = states[x], sgv = sig_vals[sg], lpv = lam_vals[lamR], gpv = g_vals[gR];
    for (int k = 0; k < ndesc; ++k) {
      const Desc& D = desc[k];
      double s = spin_of(D.src_i, D.bit_i, stx, sgv, lpv, gpv) * spin_of(D.src_j, D.bit_j, stx, sgv, lpv, gpv);
      atomicAdd(&part[k], v * s);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ndesc; k += blockDim.x) atomicAdd(&acc[desc[k].slot], part[k]);
}

// dJ = -beta acc/Z, dh = -beta acc/Z, dbeta = -(sum J <ss> + sum h <s>)
__global__ void finalize_kernel(int nE, int N, const double* acc, const double* Z, const int32_t* row_of_slot,
                                const int32_t* jn, const int32_t* hn, double denom, double beta, double* dJ, double* dh,
                                double* dbeta) {
  __shared__ double red[32];
  double H = 0;
  for (int i = threadIdx.x; i < nE + N; i += blockDim.x) {
    double ex = acc[i] / Z[row_of_slot[i]];
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

inline int nblk(long long n) { return int(std::max(1ll, std::min((n + 255) / 256, 148ll * 8))); }

template <class T>
T* to_dev(sgtn_inst* h, const std::vector<T>& v) {
  T* p = nullptr;
  SGTN_CUDA(lib_malloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) SGTN_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->st));
  return p;
}

// dense W of row r, column c: [bl][br][u][sigma]
double* densify(sgtn_inst* h, int r, int c) {
  const int C = h->M.C;
  const Column& K = h->cols[r * C + c];
  const DSite& D = h->ds[r * C + c];
  long long n = (long long)K.nBL() * K.nBR() * K.nU * K.nSig;
  double* W = dmalloc(n);
  const double* Bv = h->dB[size_t(r * C + c) * 4 + 1];
  const double* Bh = h->dB[size_t(r * C + c) * 4 + 0];
  const double* Bdr = h->dB[size_t(r * C + c) * 4 + 2];
  const double* Bdl;
  int bdl_nb;
  if (c + 1 < C) {
    Bdl = h->dB[size_t(r * C + c + 1) * 4 + 3];
    bdl_nb = K.bdl_nb;
  } else {
    double* one = h->ws.get<double>("unit_scalar", 1);
    fill(one, 1, 1.0, h->st);
    Bdl = one;
    bdl_nb = 1;
  }
  densify_kernel<<<nblk(n), 256, 0, h->st>>>(W, K.d, K.nG, K.nU, K.nSig, K.nLR, K.nGR, D.w, K.lam_x, K.u_x, K.pd_x,
                                             K.pr_x, K.pdr_x, K.s_pu, K.s_pul, K.s_pur, K.l_pl, K.l_pdl, Bv, K.bv_nb,
                                             Bh, K.bh_nb, Bdl, bdl_nb, Bdr, K.bdr_nb, n);
  ++g_count.launches;
  return W;
}

void free_all(std::vector<double*>& v) {
  for (auto& p : v) dfree(p);
  v.clear();
}

}  // namespace

namespace detail {

// Theta[(bl, chl), (out, kp)] = sum W[bl][br][out][in] A[in][chl][chr] K[br][chr][kp]
double* theta_dense(RowCtx& X, int c, const double* K, int kp) {
  sgtn_inst* h = X.h;
  cudaStream_t st = h->st;
  const Column& col = X.col(c);
  int nbl = col.nBL(), nbr = col.nBR(), nout = X.nout(c), nin = X.nin(c), chl = X.chl(c), chr = X.chr(c);
  double* Kp = h->ws.get<double>("td_Kp", size_t(chr) * nbr * kp);
  permute3(K, nbr, chr, kp, Kp, st);
  double* P = h->ws.get<double>("td_P", size_t(nin) * chl * nbr * kp);
  gemm(X.A->t[c], false, chr, Kp, false, (long long)nbr * kp, P, (long long)nbr * kp, nin * chl, nbr * kp, chr, 1.0, 0,
       st);
  double* Pp = h->ws.get<double>("td_Pp", size_t(nin) * chl * nbr * kp);
  {
    int dims[4] = {nin, chl, nbr, kp}, perm[4] = {2, 0, 1, 3};
    permute_nd(P, 4, dims, perm, Pp, st);
  }
  double* Wm = h->ws.get<double>("td_Wm", size_t(nbl) * nbr * nout * nin);
  {
    int dims[4] = {nbl, nbr, nout, nin}, perm[4] = {0, 2, 1, 3};
    permute_nd(X.Wd[c], 4, dims, perm, Wm, st);
  }
  double* T1 = h->ws.get<double>("td_T1", size_t(nbl) * nout * chl * kp);
  gemm(Wm, false, (long long)nbr * nin, Pp, false, (long long)chl * kp, T1, (long long)chl * kp, nbl * nout, chl * kp,
       nbr * nin, 1.0, 0, st);
  double* Th = h->ws.get<double>("theta", size_t(nbl) * chl * nout * kp);
  {
    int dims[4] = {nbl, nout, chl, kp}, perm[4] = {0, 2, 1, 3};
    permute_nd(T1, 4, dims, perm, Th, st);
  }
  return Th;
}

// Lnext[b][br][chr] = sum L[a][bl][chl] phi[a][out][b] W[bl][br][out][in] A[in][chl][chr]
double* update_L_dense(RowCtx& X, int c, const double* L, const Ten& phi) {
  sgtn_inst* h = X.h;
  cudaStream_t st = h->st;
  const Column& col = X.col(c);
  int nbl = col.nBL(), nbr = col.nBR(), nout = X.nout(c), nin = X.nin(c), chl = X.chl(c), chr = X.chr(c);
  long long nob = (long long)nout * phi.b;
  double* N = h->ws.get<double>("ld_N", size_t(nob) * nbl * chl);
  gemm(phi.p, true, nob, L, false, (long long)nbl * chl, N, (long long)nbl * chl, int(nob), nbl * chl, phi.a, 1.0, 0,
       st);
  double* WA = h->ws.get<double>("ld_WA", size_t(nbl) * nbr * nout * chl * chr);
  gemm(X.Wd[c], false, nin, X.A->t[c], false, (long long)chl * chr, WA, (long long)chl * chr, nbl * nbr * nout,
       chl * chr, nin, 1.0, 0, st);
  double* WAp = h->ws.get<double>("ld_WAp", size_t(nbl) * nbr * nout * chl * chr);
  {
    int dims[5] = {nbl, nbr, nout, chl, chr}, perm[5] = {2, 0, 3, 1, 4};
    permute_nd(WA, 5, dims, perm, WAp, st);
  }
  double* Np = h->ws.get<double>("ld_Np", size_t(nob) * nbl * chl);
  {
    int dims[4] = {nout, phi.b, nbl, chl}, perm[4] = {1, 0, 2, 3};
    permute_nd(N, 4, dims, perm, Np, st);
  }
  double* Ln = dmalloc((long long)phi.b * nbr * chr);
  gemm(Np, false, (long long)nout * nbl * chl, WAp, false, (long long)nbr * chr, Ln, (long long)nbr * chr, phi.b,
       nbr * chr, nout * nbl * chl, 1.0, 0, st);
  return Ln;
}

}  // namespace detail

void logz_grad(sgtn_inst* h, double* dJ, double* dh, double* dbeta) {
  if (!h->boundary_ok) throw SgtnError(-2, "contract_boundary must run first");
  if (h->n_sweeps < 1) throw SgtnError(-1, "gradients need n_sweeps >= 1 in contract_boundary");
  const int R = h->M.R, C = h->M.C, N = h->M.N;
  const int nE = int(h->M.ei.size());
  cudaStream_t st = h->st;
  // dense columns of every row, and the bound on their size
  std::vector<std::vector<double*>> W(R);
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) {
      const Column& K = h->cols[r * C + c];
      long long n = (long long)K.nBL() * K.nBR() * K.nU * K.nSig;
      if (n > (1ll << 26)) throw SgtnError(-1, "logz_grad: column tensor too large for the dense gradient path");
      W[r].push_back(densify(h, r, c));
    }
  // top-down upper boundary MPSs E_0..E_{R-1}
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
    X.dense = true;
    X.transposed = true;
    for (int c = 0; c < C; ++c) {
      const Column& K = h->cols[r * C + c];
      double* Wt = dmalloc((long long)K.nBL() * K.nBR() * K.nU * K.nSig);
      int dims[4] = {K.nBL(), K.nBR(), K.nU, K.nSig}, perm[4] = {0, 1, 3, 2};
      permute_nd(W[r][c], 4, dims, perm, Wt, st);
      X.Wd.push_back(Wt);
    }
    row_step_ctx(X, E[r], h->chi, h->n_sweeps, E[r + 1], worst);
    free_all(X.Wd);
  }
  // accumulators: slots [edges | spins], one Z per row
  double* acc = dmalloc(nE + N);
  double* Z = dmalloc(R);
  SGTN_CUDA(cudaMemsetAsync(acc, 0, (nE + N) * sizeof(double), st));
  SGTN_CUDA(cudaMemsetAsync(Z, 0, R * sizeof(double), st));
  std::vector<int32_t> row_of_slot(nE + N, 0);
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
    if (ri > rj || (ri == rj && ci > cj) ) {
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
    row_of_slot[e] = owner_r;
  }
  for (int s = 0; s < R * C; ++s) {
    const HSite& S = h->M.sites[s];
    for (size_t j = 0; j < S.spins.size(); ++j) {
      desc[s].push_back({1, int(j), 0, 0, nE + S.spins[j]});
      row_of_slot[nE + S.spins[j]] = s / C;
    }
  }
  int32_t* d_row = to_dev(h, row_of_slot);
  // per-row sandwich
  for (int r = 0; r < R; ++r) {
    RowCtx X;
    X.h = h;
    X.r = r;
    X.dense = true;
    X.transposed = false;
    X.Wd = W[r];
    X.A = &h->psi[r];
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
    for (int c = C - 1; c > 0; --c) {
      double* Th = theta_of(X, c, Re[c], bra[c].b);
      Re[c - 1] = update_R(X, c, Th, bra[c]);
    }
    Le[0] = dmalloc(1);
    fill(Le[0], 1, 1.0, st);
    for (int c = 0; c + 1 < C; ++c) Le[c + 1] = update_L(X, c, Le[c], bra[c]);
    for (int c = 0; c < C; ++c) {
      const Column& K = X.col(c);
      int nbl = K.nBL(), nbr = K.nBR(), nU = K.nU, nSig = K.nSig, chl = X.chl(c), chr = X.chr(c);
      int a = bra[c].a, ap = bra[c].b;
      // M[(bl,u),(br,sigma)] = sum L[a][bl][chl] E[a][u][a'] A[sigma][chl][chr] R[br][chr][a']
      double* Xm = dmalloc((long long)nbl * chl * nU * ap);
      gemm(Le[c], true, (long long)nbl * chl, bra[c].p, false, (long long)nU * ap, Xm, (long long)nU * ap, nbl * chl,
           nU * ap, a, 1.0, 0, st);
      double* Rp = dmalloc((long long)chr * nbr * ap);
      permute3(Re[c], nbr, chr, ap, Rp, st);
      double* AR = dmalloc((long long)nSig * chl * nbr * ap);
      gemm(h->psi[r].t[c], false, chr, Rp, false, (long long)nbr * ap, AR, (long long)nbr * ap, nSig * chl, nbr * ap,
           chr, 1.0, 0, st);
      double* Xp = dmalloc((long long)nbl * chl * nU * ap);
      {
        int dims[4] = {nbl, chl, nU, ap}, perm[4] = {0, 2, 1, 3};
        permute_nd(Xm, 4, dims, perm, Xp, st);
      }
      double* ARp = dmalloc((long long)nSig * chl * nbr * ap);
      {
        int dims[4] = {nSig, chl, nbr, ap}, perm[4] = {1, 3, 2, 0};
        permute_nd(AR, 4, dims, perm, ARp, st);
      }
      double* M = dmalloc((long long)nbl * nU * nbr * nSig);
      gemm(Xp, false, (long long)chl * ap, ARp, false, (long long)nbr * nSig, M, (long long)nbr * nSig, nbl * nU,
           nbr * nSig, chl * ap, 1.0, 0, st);
      // descriptors of this column (+ Z at column 0)
      std::vector<Desc> dv = desc[r * C + c];
      if (c == 0) dv.push_back({0, 0, 0, 0, -1});
      double* accz = dmalloc(int(dv.size()));
      SGTN_CUDA(cudaMemsetAsync(accz, 0, dv.size() * sizeof(double), st));
      std::vector<Desc> loc(dv.size());
      for (size_t k = 0; k < dv.size(); ++k) {
        loc[k] = dv[k];
        loc[k].slot = int(k);
      }
      Desc* dd = nullptr;
      SGTN_CUDA(lib_malloc(&dd, std::max<size_t>(1, loc.size()) * sizeof(Desc)));
      if (!loc.empty())
        SGTN_CUDA(cudaMemcpyAsync(dd, loc.data(), loc.size() * sizeof(Desc), cudaMemcpyHostToDevice, st));
      const HSite& S = h->M.sites[r * C + c];
      const HSite* below = h->M.site(r + 1, c);
      const HSite* right = h->M.site(r, c + 1);
      const HSite* br_ = h->M.site(r + 1, c + 1);
      std::vector<int64_t> zero1(1, 0);
      int64_t* st_d = to_dev(h, S.states);
      int64_t* sg_d = to_dev(h, below ? below->U.vals : zero1);
      int64_t* lp_d = to_dev(h, right ? right->Lam.vals : zero1);
      int64_t* gp_d = to_dev(h, br_ ? br_->proj[DUL].vals : zero1);
      const double* Bv = h->dB[size_t(r * C + c) * 4 + 1];
      const double* Bh = h->dB[size_t(r * C + c) * 4 + 0];
      const double* Bdr = h->dB[size_t(r * C + c) * 4 + 2];
      const double* Bdl;
      int bdl_nb;
      if (c + 1 < C) {
        Bdl = h->dB[size_t(r * C + c + 1) * 4 + 3];
        bdl_nb = K.bdl_nb;
      } else {
        double* one = h->ws.get<double>("unit_scalar", 1);
        fill(one, 1, 1.0, st);
        Bdl = one;
        bdl_nb = 1;
      }
      const DSite& D = h->ds[r * C + c];
      long long ncomb = (long long)K.d * nSig * nbr;
      if (!loc.empty()) {
        edge_sum_kernel<<<nblk(ncomb), 256, loc.size() * sizeof(double), st>>>(
            K.d, K.nG, nU, nSig, K.nLR, K.nGR, M, D.w, K.lam_x, K.u_x, K.pd_x, K.pr_x, K.pdr_x, K.s_pu, K.s_pul, K.s_pur,
            K.l_pl, K.l_pdl, Bv, K.bv_nb, Bh, K.bh_nb, Bdl, bdl_nb, Bdr, K.bdr_nb, st_d, sg_d, lp_d, gp_d,
            int(loc.size()), dd, accz);
        ++g_count.launches;
      }
      // scatter the column's sums into the global slots (Z of the row from column 0)
      std::vector<double> hz(loc.size());
      SGTN_CUDA(cudaMemcpyAsync(hz.data(), accz, loc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      h->sync();
      for (size_t k = 0; k < dv.size(); ++k) {
        if (dv[k].slot < 0) {
          SGTN_CUDA(cudaMemcpyAsync(Z + r, accz + k, sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
          copy(acc + dv[k].slot, accz + k, 1, st);
        }
      }
      h->sync();
      cudaFree(dd);
      cudaFree(st_d);
      cudaFree(sg_d);
      cudaFree(lp_d);
      cudaFree(gp_d);
      dfree(accz);
      dfree(Xm);
      dfree(Rp);
      dfree(AR);
      dfree(Xp);
      dfree(ARp);
      dfree(M);
    }
    for (auto& t : bra) dfree(t.p);
    free_all(Re);
    free_all(Le);
  }
  // outputs
  double *ddJ = dmalloc(std::max(nE, 1)), *ddh = dmalloc(N), *ddb = dmalloc(1);
  int32_t* jn = to_dev(h, h->M.jn.empty() ? std::vector<int32_t>(1, 0) : h->M.jn);
  int32_t* hn = to_dev(h, h->M.hn);
  finalize_kernel<<<1, 1024, 0, st>>>(nE, N, acc, Z, d_row, jn, hn, double(h->M.denom), h->beta, ddJ, ddh, ddb);
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
  dfree(Z);
  cudaFree(jn);
  cudaFree(hn);
  cudaFree(d_row);
  for (auto& m : E) free_mps(m);
  for (auto& v : W) free_all(v);
}

}  // namespace sgtn
