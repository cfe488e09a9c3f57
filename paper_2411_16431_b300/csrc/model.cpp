// Host-side clustering of an Ising instance into a generalized Potts model,
// paper Sec. III, Eqs. (2)-(4).  Written independently of any other
// implementation: states are bit patterns over a site's spins (bit 0 = +1),
// a projector class is a distinct restriction of a state to the spins that
// couple toward one neighbour, numbered in increasing pattern order.
#include <algorithm>
#include <map>
#include <unordered_map>

#include "model.h"

namespace sgtn {

static int64_t restrict_bits(int64_t x, const std::vector<int>& bits) {
  int64_t v = 0;
  for (size_t j = 0; j < bits.size(); ++j) v |= ((x >> bits[j]) & 1LL) << j;
  return v;
}

static Proj make_proj(const std::vector<int64_t>& states, const std::vector<int>& bits) {
  Proj P;
  P.bits = bits;
  std::vector<int64_t> v(states.size());
  for (size_t i = 0; i < states.size(); ++i) v[i] = restrict_bits(states[i], bits);
  P.vals = v;
  std::sort(P.vals.begin(), P.vals.end());
  P.vals.erase(std::unique(P.vals.begin(), P.vals.end()), P.vals.end());
  P.of_state.resize(states.size());
  for (size_t i = 0; i < states.size(); ++i)
    P.of_state[i] = int32_t(std::lower_bound(P.vals.begin(), P.vals.end(), v[i]) - P.vals.begin());
  P.n = int(P.vals.size());
  if (P.n == 0) P.n = 1;
  return P;
}

// class in `sub` of every class of `joint` (sub.bits must be a subset of joint.bits)
static std::vector<int32_t> component(const Proj& joint, const Proj& sub) {
  std::vector<int> pos;
  for (int b : sub.bits) pos.push_back(int(std::find(joint.bits.begin(), joint.bits.end(), b) - joint.bits.begin()));
  std::vector<int32_t> out(joint.vals.size());
  for (size_t i = 0; i < joint.vals.size(); ++i) {
    int64_t v = 0;
    for (size_t j = 0; j < pos.size(); ++j) v |= ((joint.vals[i] >> pos[j]) & 1LL) << j;
    out[i] = int32_t(std::lower_bound(sub.vals.begin(), sub.vals.end(), v) - sub.vals.begin());
  }
  return out;
}

static std::vector<int> merged(std::initializer_list<const std::vector<int>*> ls) {
  std::vector<int> o;
  for (auto* l : ls) o.insert(o.end(), l->begin(), l->end());
  std::sort(o.begin(), o.end());
  o.erase(std::unique(o.begin(), o.end()), o.end());
  return o;
}

std::string Model::build(int32_t n_spins, int64_t n_edges, const int32_t* ei_, const int32_t* ej_,
                         const int32_t* j_num, const int32_t* h_num, int32_t denom_,
                         const int32_t* site_of_spin_, int32_t rows, int32_t cols,
                         const int64_t* state_offsets, const int64_t* states) {
  if (n_spins <= 0 || n_edges < 0 || rows <= 0 || cols <= 0 || denom_ <= 0) return "bad sizes";
  if ((n_edges > 0 && (!ei_ || !ej_ || !j_num)) || !h_num || !site_of_spin_) return "null input array";
  if ((state_offsets == nullptr) != (states == nullptr)) return "state_offsets and states must both be set or both NULL";
  R = rows;
  C = cols;
  N = n_spins;
  denom = denom_;
  ei.assign(ei_, ei_ + n_edges);
  ej.assign(ej_, ej_ + n_edges);
  jn.assign(j_num, j_num + n_edges);
  hn.assign(h_num, h_num + n_spins);
  site_of_spin.assign(site_of_spin_, site_of_spin_ + n_spins);
  sites.assign(R * C, HSite());
  for (int s = 0; s < R * C; ++s) {
    sites[s].r = s / C;
    sites[s].c = s % C;
  }
  for (int i = 0; i < N; ++i) {
    int s = site_of_spin[i];
    if (s < 0 || s >= R * C) return "site_of_spin out of range";
    sites[s].spins.push_back(i);  // increasing i
  }
  std::vector<int> local(N);
  for (auto& S : sites)
    for (size_t j = 0; j < S.spins.size(); ++j) local[S.spins[j]] = int(j);
  for (int s = 0; s < R * C; ++s) {
    HSite& S = sites[s];
    int k = int(S.spins.size());
    if (states) {
      int64_t a = state_offsets[s], b = state_offsets[s + 1];
      if (b <= a) return "empty state list";
      S.states.assign(states + a, states + b);
      for (int64_t x : S.states)
        if (x < 0 || (k < 63 && (x >> k) != 0)) return "state pattern outside the site's spins";
      std::vector<int64_t> chk = S.states;
      std::sort(chk.begin(), chk.end());
      if (std::adjacent_find(chk.begin(), chk.end()) != chk.end()) return "duplicate state in list";
    } else {
      if (k > 16) return "site with more than 16 spins needs an explicit state list";
      S.states.resize(size_t(1) << k);
      for (int64_t x = 0; x < (int64_t(1) << k); ++x) S.states[x] = x;
    }
    S.d = int(S.states.size());
    S.E.assign(S.d, 0);
    for (int j = 0; j < k; ++j) {
      int64_t h = hn[S.spins[j]];
      for (int x = 0; x < S.d; ++x) S.E[x] += h * (1 - 2 * ((S.states[x] >> j) & 1));
    }
  }
  // edges: intra-site energies or inter-site coupled bit sets
  std::map<std::pair<int, int>, std::vector<int64_t>> pair_edges;  // (a<b) -> list of edge ids
  for (int64_t e = 0; e < n_edges; ++e) {
    int i = ei[e], j = ej[e];
    if (i < 0 || j < 0 || i >= N || j >= N || i == j) return "bad edge";
    int si = site_of_spin[i], sj = site_of_spin[j];
    if (si == sj) {
      HSite& S = sites[si];
      int a = local[i], b = local[j];
      for (int x = 0; x < S.d; ++x)
        S.E[x] += int64_t(jn[e]) * (1 - 2 * ((S.states[x] >> a) & 1)) * (1 - 2 * ((S.states[x] >> b) & 1));
    } else {
      int ra = si / C, ca = si % C, rb = sj / C, cb = sj % C;
      if (std::max(std::abs(ra - rb), std::abs(ca - cb)) != 1) return "coupled clusters are not grid neighbours";
      pair_edges[{std::min(si, sj), std::max(si, sj)}].push_back(e);
    }
  }
  for (auto& S : sites) S.Emin = S.d ? *std::min_element(S.E.begin(), S.E.end()) : 0;
  for (auto& S : sites) {
    int me = S.r * C + S.c;
    for (int d = 0; d < 8; ++d) {
      int rr = S.r + kDr[d], cc = S.c + kDc[d];
      std::vector<int> bits;
      if (rr >= 0 && rr < R && cc >= 0 && cc < C) {
        int t = rr * C + cc;
        auto it = pair_edges.find({std::min(me, t), std::max(me, t)});
        if (it != pair_edges.end())
          for (int64_t e : it->second) {
            int mine = site_of_spin[ei[e]] == me ? ei[e] : ej[e];
            bits.push_back(local[mine]);
          }
      }
      std::sort(bits.begin(), bits.end());
      bits.erase(std::unique(bits.begin(), bits.end()), bits.end());
      S.coupled[d] = bits;
      S.proj[d] = make_proj(S.states, bits);
    }
    S.U = make_proj(S.states, merged({&S.coupled[DU], &S.coupled[DUL], &S.coupled[DUR]}));
    S.Lam = make_proj(S.states, merged({&S.coupled[DL_], &S.coupled[DDL]}));
    S.Xk = make_proj(S.states, merged({&S.coupled[DR_], &S.coupled[DD], &S.coupled[DDL], &S.coupled[DDR]}));
    S.U_u = component(S.U, S.proj[DU]);
    S.U_ul = component(S.U, S.proj[DUL]);
    S.U_ur = component(S.U, S.proj[DUR]);
    S.Lam_l = component(S.Lam, S.proj[DL_]);
    S.Lam_dl = component(S.Lam, S.proj[DDL]);
  }
  // compressed inter-cluster energies for the forward directions R, D, DR, DL
  tab.assign(size_t(R) * C * 4, HTable());
  const Dir fwd[4] = {DR_, DD, DDR, DDL};
  for (auto& S : sites) {
    int me = S.r * C + S.c;
    for (int k = 0; k < 4; ++k) {
      Dir d = fwd[k];
      HTable& T = tab[size_t(me) * 4 + k];
      const HSite* O = site(S.r + kDr[d], S.c + kDc[d]);
      if (!O) {
        T.E.assign(1, 0);
        continue;
      }
      const Proj& PS = S.proj[d];
      const Proj& PT = O->proj[kOpp[d]];
      T.nA = PS.n;
      T.nB = PT.n;
      T.E.assign(size_t(T.nA) * T.nB, 0);
      int them = O->r * C + O->c;
      auto it = pair_edges.find({std::min(me, them), std::max(me, them)});
      if (it != pair_edges.end())
        for (int64_t e : it->second) {
          int mine = site_of_spin[ei[e]] == me ? ei[e] : ej[e];
          int theirs = mine == ei[e] ? ej[e] : ei[e];
          int bs = int(std::find(PS.bits.begin(), PS.bits.end(), local[mine]) - PS.bits.begin());
          int bt = int(std::find(PT.bits.begin(), PT.bits.end(), local[theirs]) - PT.bits.begin());
          for (int a = 0; a < T.nA; ++a) {
            int64_t sa = 1 - 2 * ((PS.vals[a] >> bs) & 1);
            for (int b = 0; b < T.nB; ++b) {
              int64_t sb = 1 - 2 * ((PT.vals[b] >> bt) & 1);
              T.E[size_t(a) * T.nB + b] += int64_t(jn[e]) * sa * sb;
            }
          }
        }
      T.Emin = *std::min_element(T.E.begin(), T.E.end());
    }
  }
  return "";
}

}  // namespace sgtn
