// Internal data model of the sgtn library (not part of the C ABI).
//
// Host side: clustering of spins into Potts sites (paper Sec. III, Eqs. 2-4).
// Device side: per-site index tables, per-beta weights, per-column term
// tables that drive the sparse "site diagram" contractions of Fig. 7.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace sgtn {

// neighbour directions of a site
enum Dir { DR_ = 0, DL_ = 1, DD = 2, DU = 3, DDR = 4, DDL = 5, DUR = 6, DUL = 7 };
// DR_ = right (0,+1), DL_ = left (0,-1), DD = down, DU = up, DDR = down-right,
// DDL = down-left, DUR = up-right, DUL = up-left
static const int kDr[8] = {0, 0, 1, -1, 1, 1, -1, -1};
static const int kDc[8] = {1, -1, 0, 0, 1, -1, 1, -1};
static const int kOpp[8] = {DL_, DR_, DU, DD, DUL, DUR, DDL, DDR};

// Classes of the restriction of a site's states to a set of its spins.
struct Proj {
  std::vector<int> bits;           // local bit positions, increasing
  std::vector<int64_t> vals;       // distinct restricted patterns, increasing
  std::vector<int32_t> of_state;   // class index of every state
  int n = 1;
};

struct HSite {
  int r = 0, c = 0;
  std::vector<int> spins;          // global ids, increasing
  std::vector<int64_t> states;     // bit patterns
  int d = 0;
  std::vector<int64_t> E;          // intra-cluster energy numerators
  int64_t Emin = 0;
  std::vector<int> coupled[8];
  Proj proj[8];
  Proj U;                          // up exposure: u, ul, ur
  Proj Lam;                        // left exposure: l, dl
  Proj Xk;                         // merge class: r, d, dl, dr
  std::vector<int32_t> U_u, U_ul, U_ur, Lam_l, Lam_dl;
};

struct HTable {                    // compressed energies of a coupled pair, Eq. (3)
  int nA = 1, nB = 1;
  std::vector<int64_t> E;          // [nA][nB]
  int64_t Emin = 0;
};

// device buffer helper
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  void free_() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Term table of a segmented gathered GEMM:
//   O[seg] = sum_{t in seg} coef[t] * X[xoff(t)] * Y[yoff(t)]   (blocks)
// with xoff = xr*xrs + xc*xcs, yoff = yr*yrs + yc*ycs, ooff = orow*ors + ocol*ocs
struct TermTable {
  int nseg = 0, nterm = 0;
  std::vector<int32_t> h_seg_ptr, h_seg_or, h_seg_oc;
  std::vector<int32_t> h_xr, h_xc, h_yr, h_yc, h_cidx, h_csrow;
  int32_t *seg_ptr = nullptr, *seg_or = nullptr, *seg_oc = nullptr;
  int32_t *xr = nullptr, *xc = nullptr, *yr = nullptr, *yc = nullptr, *cidx = nullptr, *csrow = nullptr;
  // balanced split for the GEMM (nvseg = 0: none): virtual segment v covers
  // terms [vseg_ptr[v], vseg_ptr[v+1]); segment s owns virtual segments
  // [vfirst[s], vfirst[s+1])
  int nvseg = 0;
  int32_t *vseg_ptr = nullptr, *vfirst = nullptr;
};

// Static description of MPO column c of row r (see the boundary code for the
// index conventions) and its device tables.
struct Column {
  int r = 0, c = 0;
  int d = 1;
  int nLam = 1, nG = 1, nU = 1, nSig = 1, nLR = 1, nGR = 1;
  int nPd = 1, nPr = 1, nPdr = 1, nE = 1;
  int nBL() const { return nLam * nG; }
  int nBR() const { return nLR * nGR; }
  int nA() const { return nPd * nE * nG; }     // projected-MPS blocks (pd, e, g)
  int nK() const { return nPr * nE * nPdr; }   // absorbed connecting-tensor blocks (pr, e, pdr)
  // per-state classes (device, int32[d])
  int32_t *lam_x = nullptr, *u_x = nullptr, *pd_x = nullptr, *pr_x = nullptr, *pdr_x = nullptr;
  // per sigma class (site below): components u, ul, ur
  int32_t *s_pu = nullptr, *s_pul = nullptr, *s_pur = nullptr;
  // per right-bond lambda' class (site right): components l, dl
  int32_t *l_pl = nullptr, *l_pdl = nullptr;
  // table shapes for the four bond factors touching this column
  int bv_nb = 1, bh_nb = 1, bdl_na = 1, bdl_nb = 1, bdr_nb = 1;
  TermTable theta;   // segments (bl, u), terms (x, e)
  TermTable lupd;    // segments (pr, e, pdr), terms (x, g)
  TermTable bs_rows; // block-sparse Theta grouped by row block bl: terms (xr = seg, yr = u)
  TermTable bs_cols; // grouped by column block u: terms (xr = seg, xc = bl, yr = bl, yc = seg)
  TermTable renv;    // segments bl, terms (x, e), column scale row = u
  // the (u, bl) pairs that lupd terms read, one segment each (xr = u, yr = bl),
  // and per lupd term the index of its pair
  TermTable lpairs;
  int32_t* lupd_pair = nullptr;
  // per-beta dense weight matrices (device, double)
  double* Wa = nullptr;   // [nA][nSig]
  double* Wk = nullptr;   // [nK][nBR]
};

// Tables of the gradient path, built on its first call.  tcols[r*C + c]
// (rows 0..R-2) is the transposed row MPO T_r^T written as a forward-form
// column over virtual states y = (x, sigma); xl / msig / pair_x index the
// environment correlators of column r*C + c.
struct GradTables {
  bool built = false;
  std::vector<Column> tcols;
  std::vector<double*> tw, tbh;    // per virtual state weights, horizontal tables Bh' (per beta)
  std::vector<int> npur;           // classes of the site below toward the right neighbour
  std::vector<TermTable> xl;       // one segment per ((lam, u) pair, g)
  std::vector<TermTable> msig;     // one segment per sigma
  std::vector<int32_t*> pair_x;    // (lam, u) pair of every state
  std::vector<int> npairs;
  std::vector<int> texp, tlexp;    // weight exponents of the transposed columns (Theta, left updates)
};

struct MPS {
  int C = 0;
  std::vector<int> phys, bond;     // phys[C], bond[C+1]
  std::vector<double*> t;          // [phys][bond_l][bond_r] per column
  double lognorm = 0.0;
  bool valid = false;
};

struct Model {
  int R = 0, C = 0, N = 0, denom = 1;
  std::vector<int32_t> ei, ej, jn, hn, site_of_spin;
  std::vector<HSite> sites;
  std::vector<HTable> tab;         // [site*4 + k], k: 0=R, 1=D, 2=DR, 3=DL
  static int tab_slot(Dir d) { return d == DR_ ? 0 : d == DD ? 1 : d == DDR ? 2 : d == DDL ? 3 : -1; }
  const HSite* site(int r, int c) const {
    return (r >= 0 && r < R && c >= 0 && c < C) ? &sites[r * C + c] : nullptr;
  }
  std::string build(int32_t n_spins, int64_t n_edges, const int32_t* ei, const int32_t* ej,
                    const int32_t* j_num, const int32_t* h_num, int32_t denom,
                    const int32_t* site_of_spin, int32_t rows, int32_t cols,
                    const int64_t* state_offsets, const int64_t* states);
};

}  // namespace sgtn
