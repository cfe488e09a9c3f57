// Device-side set-up: per-site index tables, per-column term tables of the
// sparse site diagrams (Fig. 7), and the per-beta Boltzmann factors (Eq. 5).
#include <algorithm>
#include <map>
#include <numeric>
#include <tuple>

#include "handle.h"

namespace sgtn {

namespace {

// Group terms by segment key and upload.
struct TermBuilder {
  struct T {
    int64_t key;
    int32_t sor, soc, xr, xc, yr, yc, cidx, csrow;
  };
  std::vector<T> v;
  void add(int64_t key, int sor, int soc, int xr, int xc, int yr, int yc, int cidx, int csrow) {
    v.push_back({key, sor, soc, xr, xc, yr, yc, cidx, csrow});
  }
  void finish(sgtn_inst* h, TermTable& tt) {
    std::stable_sort(v.begin(), v.end(), [](const T& a, const T& b) { return a.key < b.key; });
    tt.h_seg_ptr.clear();
    for (size_t i = 0; i < v.size(); ++i) {
      if (i == 0 || v[i].key != v[i - 1].key) {
        tt.h_seg_ptr.push_back(int32_t(i));
        tt.h_seg_or.push_back(v[i].sor);
        tt.h_seg_oc.push_back(v[i].soc);
      }
      tt.h_xr.push_back(v[i].xr);
      tt.h_xc.push_back(v[i].xc);
      tt.h_yr.push_back(v[i].yr);
      tt.h_yc.push_back(v[i].yc);
      tt.h_cidx.push_back(v[i].cidx);
      tt.h_csrow.push_back(v[i].csrow);
    }
    tt.h_seg_ptr.push_back(int32_t(v.size()));
    tt.nseg = int(tt.h_seg_ptr.size()) - 1;
    tt.nterm = int(v.size());
    tt.seg_ptr = h->upload(tt.h_seg_ptr);
    tt.seg_or = h->upload(tt.h_seg_or);
    tt.seg_oc = h->upload(tt.h_seg_oc);
    tt.xr = h->upload(tt.h_xr);
    tt.xc = h->upload(tt.h_xc);
    tt.yr = h->upload(tt.h_yr);
    tt.yc = h->upload(tt.h_yc);
    tt.cidx = h->upload(tt.h_cidx);
    tt.csrow = h->upload(tt.h_csrow);
    // segments much longer than nterm / (2 x 148) are cut into equal parts so
    // that one GEMM launch has no straggler CTA
    const int chunk = std::max(2, (tt.nterm + 295) / 296);
    std::vector<int32_t> vptr, vfirst;
    for (int g = 0; g < tt.nseg; ++g) {
      const int b = tt.h_seg_ptr[g], e = tt.h_seg_ptr[g + 1], len = e - b;
      const int parts = std::max(1, (len + chunk - 1) / chunk), step = (len + parts - 1) / parts;
      vfirst.push_back(int32_t(vptr.size()));
      for (int x = b; x < e; x += step) vptr.push_back(x);
    }
    vfirst.push_back(int32_t(vptr.size()));
    vptr.push_back(tt.nterm);
    if (int(vfirst.back()) > tt.nseg) {
      tt.nvseg = vfirst.back();
      tt.vseg_ptr = h->upload(vptr);
      tt.vfirst = h->upload(vfirst);
    }
    v.clear();
    v.shrink_to_fit();
  }
};

}  // namespace

// Term tables of a column from its per-state classes (Lam x, U x, pd x, pr x,
// pdr x; the column's class counts must be set): the site diagram (segments
// (bl, u), terms (x, g, e)), the right-environment form (segments bl), the
// left-environment update (segments (pr, e, pdr)) with its (u, bl) pairs, and
// the block-sparse groupings of the site-diagram output.
void build_column_tables(sgtn_inst* h, Column& K, const std::vector<int32_t>& lam, const std::vector<int32_t>& u,
                         const std::vector<int32_t>& pd, const std::vector<int32_t>& pr,
                         const std::vector<int32_t>& pdr) {
  const int d = int(lam.size());
  TermBuilder tb;
  for (int x = 0; x < d; ++x)
    for (int g = 0; g < K.nG; ++g)
      for (int e = 0; e < K.nE; ++e) {
        int bl = lam[x] * K.nG + g;
        int ablk = (pd[x] * K.nE + e) * K.nG + g;
        int kblk = (pr[x] * K.nE + e) * K.nPdr + pdr[x];
        tb.add(int64_t(bl) * K.nU + u[x], bl, u[x], ablk, 0, kblk, 0, x, u[x]);
      }
  tb.finish(h, K.theta);
  for (int x = 0; x < d; ++x)
    for (int g = 0; g < K.nG; ++g)
      for (int e = 0; e < K.nE; ++e) {
        int bl = lam[x] * K.nG + g;
        int ablk = (pd[x] * K.nE + e) * K.nG + g;
        int kblk = (pr[x] * K.nE + e) * K.nPdr + pdr[x];
        tb.add(bl, bl, 0, ablk, 0, kblk, 0, x, u[x]);
      }
  tb.finish(h, K.renv);
  for (int x = 0; x < d; ++x)
    for (int g = 0; g < K.nG; ++g)
      for (int e = 0; e < K.nE; ++e) {
        int bl = lam[x] * K.nG + g;
        int ablk = (pd[x] * K.nE + e) * K.nG + g;
        int kblk = (pr[x] * K.nE + e) * K.nPdr + pdr[x];
        tb.add(kblk, kblk, 0, u[x], bl, ablk, 0, x, u[x]);
      }
  tb.finish(h, K.lupd);
  {
    // distinct (u, bl) pairs read by the lupd terms: the left-environment
    // update forms its intermediate only for these
    std::map<std::pair<int32_t, int32_t>, int32_t> pid;
    std::vector<int32_t> tp(K.lupd.nterm);
    for (int t = 0; t < K.lupd.nterm; ++t) {
      auto key = std::make_pair(K.lupd.h_xr[t], K.lupd.h_xc[t]);
      auto it = pid.find(key);
      if (it == pid.end()) it = pid.emplace(key, int32_t(pid.size())).first;
      tp[t] = it->second;
    }
    for (auto& kv : pid) tb.add(kv.second, kv.second, 0, kv.first.first, 0, kv.first.second, 0, 0, 0);
    tb.finish(h, K.lpairs);
    K.lupd_pair = h->upload(tp);
  }
  // groupings of the site-diagram output blocks (one block per theta segment)
  for (int sg = 0; sg < K.theta.nseg; ++sg) {
    int bl = K.theta.h_seg_or[sg], uu = K.theta.h_seg_oc[sg];
    tb.add(bl, bl, 0, sg, 0, uu, 0, 0, 0);
  }
  tb.finish(h, K.bs_rows);
  for (int sg = 0; sg < K.theta.nseg; ++sg) {
    int bl = K.theta.h_seg_or[sg], uu = K.theta.h_seg_oc[sg];
    tb.add(uu, uu, 0, sg, bl, bl, sg, 0, 0);
  }
  tb.finish(h, K.bs_cols);
}

// One term per segment i (in order): block rows xr[i] of X and yr[i] of Y.
void build_pair_table(sgtn_inst* h, TermTable& tt, const std::vector<int32_t>& xr, const std::vector<int32_t>& yr) {
  TermBuilder tb;
  for (size_t i = 0; i < xr.size(); ++i) tb.add(int64_t(i), int32_t(i), 0, xr[i], 0, yr[i], 0, 0, 0);
  tb.finish(h, tt);
}

void setup_device(sgtn_inst* h) {
  Model& M = h->M;
  const int R = M.R, C = M.C;
  h->ds.resize(R * C);
  for (int s = 0; s < R * C; ++s) {
    const HSite& S = M.sites[s];
    DSite& D = h->ds[s];
    D.d = S.d;
    D.E = h->upload(S.E);
    D.w = h->dalloc<double>(S.d);
    for (int d = 0; d < 8; ++d) D.cls[d] = h->upload(S.proj[d].of_state);
    D.lam_x = h->upload(S.Lam.of_state);
    D.u_x = h->upload(S.U.of_state);
    D.xk_x = h->upload(S.Xk.of_state);
    D.U_u = h->upload(S.U_u);
    D.U_ul = h->upload(S.U_ul);
    D.U_ur = h->upload(S.U_ur);
    D.Lam_l = h->upload(S.Lam_l);
    D.Lam_dl = h->upload(S.Lam_dl);
  }
  h->dE.assign(size_t(R) * C * 4, nullptr);
  h->dB.assign(size_t(R) * C * 4, nullptr);
  for (size_t i = 0; i < h->dE.size(); ++i) {
    h->dE[i] = h->upload(M.tab[i].E);
    h->dB[i] = h->dalloc<double>(M.tab[i].E.size());
  }
  int maxn = 1;
  h->cols.assign(R * C, Column());
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) {
      Column& K = h->cols[r * C + c];
      const HSite& S = M.sites[r * C + c];
      const HSite* below = M.site(r + 1, c);
      const HSite* right = M.site(r, c + 1);
      const HSite* br = M.site(r + 1, c + 1);
      const DSite& D = h->ds[r * C + c];
      K.r = r;
      K.c = c;
      K.d = S.d;
      K.nLam = S.Lam.n;
      K.nU = S.U.n;
      K.nG = below ? below->proj[DUL].n : 1;
      K.nSig = below ? below->U.n : 1;
      K.nLR = right ? right->Lam.n : 1;
      K.nGR = br ? br->proj[DUL].n : 1;
      K.nPd = S.proj[DD].n;
      K.nPr = S.proj[DR_].n;
      K.nPdr = S.proj[DDR].n;
      K.nE = right ? right->proj[DDL].n : 1;
      K.lam_x = D.lam_x;
      K.u_x = D.u_x;
      K.pd_x = D.cls[DD];
      K.pr_x = D.cls[DR_];
      K.pdr_x = D.cls[DDR];
      std::vector<int32_t> zero1(1, 0);
      if (below) {
        const DSite& Db = h->ds[(r + 1) * C + c];
        K.s_pu = Db.U_u;
        K.s_pul = Db.U_ul;
        K.s_pur = Db.U_ur;
      } else {
        K.s_pu = K.s_pul = K.s_pur = h->upload(zero1);
      }
      if (right) {
        const DSite& Dr = h->ds[r * C + c + 1];
        K.l_pl = Dr.Lam_l;
        K.l_pdl = Dr.Lam_dl;
      } else {
        K.l_pl = K.l_pdl = h->upload(zero1);
      }
      K.bv_nb = M.tab[size_t(r * C + c) * 4 + 1].nB;
      K.bh_nb = M.tab[size_t(r * C + c) * 4 + 0].nB;
      K.bdr_nb = M.tab[size_t(r * C + c) * 4 + 2].nB;
      if (right) {
        K.bdl_na = M.tab[size_t(r * C + c + 1) * 4 + 3].nA;
        K.bdl_nb = M.tab[size_t(r * C + c + 1) * 4 + 3].nB;
      }
      build_column_tables(h, K, S.Lam.of_state, S.U.of_state, S.proj[DD].of_state, S.proj[DR_].of_state,
                          S.proj[DDR].of_state);
      K.Wa = h->dalloc<double>(size_t(K.nA()) * K.nSig);
      K.Wk = h->dalloc<double>(size_t(K.nK()) * K.nBR());
      maxn = std::max({maxn, S.d, K.nU, K.nSig, K.nBL(), K.nBR()});
    }
  h->iota_n = std::max(maxn, 4096);
  std::vector<int32_t> io(h->iota_n);
  std::iota(io.begin(), io.end(), 0);
  h->iota = h->upload(io);
  h->psi.assign(R, MPS());
  h->theta_exp.assign(R * C, 0);
  h->lenv_exp.assign(R * C, 0);
  h->sync();
}

void set_beta_device(sgtn_inst* h, double beta) {
  Model& M = h->M;
  const int R = M.R, C = M.C;
  const double bd = beta / double(M.denom);
  double off = 0.0;
  for (int s = 0; s < R * C; ++s) {
    boltzmann(h->ds[s].E, h->ds[s].d, M.sites[s].Emin, bd, h->ds[s].w, h->st);
    off += -bd * double(M.sites[s].Emin);
  }
  for (size_t i = 0; i < h->dE.size(); ++i) {
    boltzmann(h->dE[i], (long long)M.tab[i].E.size(), M.tab[i].Emin, bd, h->dB[i], h->st);
    off += -bd * double(M.tab[i].Emin);
  }
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) {
      Column& K = h->cols[r * C + c];
      const double* Bv = h->dB[size_t(r * C + c) * 4 + 1];
      const double* Bh = h->dB[size_t(r * C + c) * 4 + 0];
      const double* Bdr = h->dB[size_t(r * C + c) * 4 + 2];
      // Bdl couples (r, c+1) with (r+1, c); without a right neighbour it is the 1x1 table [1]
      const double* Bdl = (c + 1 < C) ? h->dB[size_t(r * C + c + 1) * 4 + 3] : h->dB[size_t(r * C + c) * 4 + 3];
      int bdl_nb = (c + 1 < C) ? K.bdl_nb : 1;
      if (c + 1 >= C) {
        // the site's own DL table is not 1x1 in general: use a unit scalar instead
        double* one = h->ws.get<double>("unit_scalar", 1);
        fill(one, 1, 1.0, h->st);
        Bdl = one;
      }
      build_Wa(K.Wa, K.nPd, K.nE, K.nG, K.nSig, K.s_pu, K.s_pul, K.s_pur, Bv, K.bv_nb, Bdl, bdl_nb, h->st);
      build_Wk(K.Wk, K.nPr, K.nE, K.nPdr, K.nLR, K.nGR, K.l_pl, K.l_pdl, Bh, K.bh_nb, Bdr, K.bdr_nb, h->st);
    }
  h->check();
  // the weights' exponents of the mixed contractions depend on beta: learn them afresh
  std::fill(h->theta_exp.begin(), h->theta_exp.end(), 0);
  std::fill(h->lenv_exp.begin(), h->lenv_exp.end(), 0);
  h->log_offset = off;
  h->beta = beta;
  h->beta_set = true;
  h->boundary_ok = false;
  h->sync();
}

void free_mps(MPS& m) {
  for (double* p : m.t) pool_free(p);
  m.t.clear();
  m.valid = false;
}

}  // namespace sgtn
