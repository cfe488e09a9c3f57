// Branch-and-bound step (paper Sec. III.A, Fig. 3) on the device.
//
// For partial configurations k (the beam) and the next cluster n = (r, c):
//  1. f_k[c'][u]  Boltzmann factors between the fixed row r-1 of branch k and
//     class u of the up exposure of (r, c')  (1 in the top row).
//  2. E_k  left environment: row r's placed columns < c contracted with
//     psi_r (Fig. 6b); F_k right environment: the unplaced columns > c summed
//     over their states with the factors f_k, contracted with psi_r.
//  3. s_k(x) = f_k[c][U x] w_x sum_{g,e} E_k[(Lam x, g)] Ahat[(pd x, e, g)] Ftil_k[(pr x, e, pdr x)]
//     and the chain rule log p = log p_k + log(s_k(x) / sum_x' s_k(x'))  (Eq. 6);
//     negative scores (possible with an approximate psi) are clamped to 0.
//  4. Merge (Eq. 7): the boundary of candidate (k, x) is the pair
//     (boundary classes of k that stay on the boundary, merge class of x);
//     the first part is turned into an exact parent class id by comparing
//     the class vectors of all branches, so the merge key is exact (no hash).
//     The most probable candidate of each key survives; ties go to the
//     lexicographically smaller configuration.
//  5. Top-M by (log p desc, configuration asc) through a radix select on the
//     ordered bits of log p; p_d = largest log p among valid candidates that
//     did not survive.
#include <algorithm>
#include <climits>
#include <cmath>
#include <deque>
#include <iterator>
#include <memory>
#include <numeric>
#include <string>
#include <type_traits>
#include <unordered_map>

#include "../../include/sgtn.h"
#include "handle.h"

namespace sgtn {

namespace {

__device__ __host__ inline unsigned long long ord_key(double v) {
  unsigned long long u;
  memcpy(&u, &v, sizeof(u));
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
constexpr double TIE_REL = 1e-10;   // log p within this (relative) count as tied
__device__ __host__ inline double tie_tol(double lp) { return TIE_REL * fmax(1.0, fabs(lp)); }
__device__ __host__ inline double key_to_double(unsigned long long k) {
  unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  double v;
  memcpy(&v, &u, sizeof(v));
  return v;
}

__global__ void upper_f_kernel(int K, int nU, int r, int cc, int C, const int32_t* cfg, int cfg_ld,
                               const int32_t* up_pd, const double* Bv, int bv_nb, const int32_t* U_u,
                               const int32_t* ul_pdr, const double* Bdr, int bdr_nb, const int32_t* U_ul,
                               const int32_t* ur_pdl, const double* Bdl, int bdl_nb, const int32_t* U_ur,
                               double* f) {
  long long n = (long long)nU * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int k = int(e % K), u = int(e / K);
    double v = 1.0;
    if (r > 0) {
      const int32_t* row = cfg + (long long)k * cfg_ld + (r - 1) * C;
      v *= Bv[(long long)up_pd[row[cc]] * bv_nb + U_u[u]];
      if (ul_pdr) v *= Bdr[(long long)ul_pdr[row[cc - 1]] * bdr_nb + U_ul[u]];
      if (ur_pdl) v *= Bdl[(long long)ur_pdl[row[cc + 1]] * bdl_nb + U_ur[u]];
    }
    f[e] = v;
  }
}

// new left environment for branch kk (parent par[kk], state xs[kk]) at column c:
// Eout[(lam',g')][ar][kk] = sum_e [pi_dl lam' = e] Bh[pr_x, pi_l lam'] Bdr[pdr_x, g'] v[e][ar],
// v[e][ar] = sum_g sum_al Ein[(lam_x, g)][al][par] Ahat[(pd_x, e, g)][al][ar]; normalised by max |.|
__global__ void lenv_kernel(int Kin, int Kout, const int32_t* par, const int32_t* xs, const double* Ein, int chl,
                            int chr, int nG, int nE, int nPdr, int nLR, int nGR, const double* Ahat,
                            const int32_t* lam_x, const int32_t* pd_x, const int32_t* pr_x, const int32_t* pdr_x,
                            const int32_t* l_pl, const int32_t* l_pdl, const double* Bh, int bh_nb, const double* Bdr,
                            int bdr_nb, double* Eout) {
  extern __shared__ double sm[];
  double* v = sm;                  // [nE][chr]
  __shared__ double red[32];
  int kk = blockIdx.x;
  int k = par[kk], x = xs[kk];
  for (int i = threadIdx.x; i < nE * chr; i += blockDim.x) {
    int e = i / chr, ar = i % chr;
    double s = 0;
    for (int g = 0; g < nG; ++g) {
      const double* A = Ahat + (((long long)pd_x[x] * nE + e) * nG + g) * chl * chr;
      const double* E = Ein + (long long)(lam_x[x] * nG + g) * chl * Kin;
      for (int al = 0; al < chl; ++al) s = fma(E[(long long)al * Kin + k], A[(long long)al * chr + ar], s);
    }
    v[i] = s;
  }
  __syncthreads();
  int nBR = nLR * nGR;
  double mx = 0;
  for (int i = threadIdx.x; i < nBR * chr; i += blockDim.x) {
    int br = i / chr, ar = i % chr;
    int lam = br / nGR, gp = br % nGR;
    double val = Bh[(long long)pr_x[x] * bh_nb + l_pl[lam]] * Bdr[(long long)pdr_x[x] * bdr_nb + gp] *
                 v[l_pdl[lam] * chr + ar];
    Eout[(long long)i * Kout + kk] = val;
    mx = fmax(mx, fabs(val));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    red[0] = m > 0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  double s = red[0];
  for (int i = threadIdx.x; i < nBR * chr; i += blockDim.x) Eout[(long long)i * Kout + kk] *= s;
}

// divide every column k of X[rows][K] by its max |.|
__global__ void colnorm_kernel(double* X, long long rows, int K) {
  int k = blockIdx.x;
  __shared__ double red[32];
  double mx = 0;
  for (long long i = threadIdx.x; i < rows; i += blockDim.x) mx = fmax(mx, fabs(X[i * K + k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    red[0] = m > 0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  double s = red[0];
  for (long long i = threadIdx.x; i < rows; i += blockDim.x) X[i * K + k] *= s;
}

// out[i][k] = in[i][anc[k]]  (rows x K from rows x K0)
__global__ void gather_cols_kernel(const double* in, long long rows, int K0, const int32_t* anc, int K, double* out) {
  const long long n = rows * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K;
    const int k = int(e % K);
    out[e] = in[i * K0 + anc[k]];
  }
}

// s[k][x] for all branches k (threads) of one state x (block)
template <class CT>
__global__ void score_kernel(int K, int d, int chl, int chr, int nG, int nE, int nPdr, const double* E,
                             const double* Ahat, const double* Ft, const double* f, const double* w,
                             const int32_t* lam_x, const int32_t* u_x, const int32_t* pd_x, const int32_t* pr_x,
                             const int32_t* pdr_x, double* s) {
  extern __shared__ unsigned char smraw[];
  CT* As = reinterpret_cast<CT*>(smraw);   // chl * chr
  int x = blockIdx.x;
  CT acc[4] = {0, 0, 0, 0};
  for (int g = 0; g < nG; ++g)
    for (int e = 0; e < nE; ++e) {
      const double* A = Ahat + (((long long)pd_x[x] * nE + e) * nG + g) * chl * chr;
      __syncthreads();
      for (int i = threadIdx.x; i < chl * chr; i += blockDim.x) As[i] = CT(A[i]);
      __syncthreads();
      const double* Eb = E + (long long)(lam_x[x] * nG + g) * chl * K;
      const double* Fb = Ft + (((long long)pr_x[x] * nE + e) * nPdr + pdr_x[x]) * chr * K;
      for (int j = 0; j < 4; ++j) {
        int k = threadIdx.x + j * blockDim.x;
        if (k >= K) break;
        CT a2 = 0;
        for (int ar = 0; ar < chr; ++ar) {
          CT t = 0;
          for (int al = 0; al < chl; ++al) t = fma(CT(Eb[(long long)al * K + k]), As[al * chr + ar], t);
          a2 = fma(t, CT(Fb[(long long)ar * K + k]), a2);
        }
        acc[j] += a2;
      }
    }
  for (int j = 0; j < 4; ++j) {
    int k = threadIdx.x + j * blockDim.x;
    if (k >= K) break;
    s[(long long)k * d + x] = f[(long long)u_x[x] * K + k] * w[x] * double(acc[j]);
  }
}

// Same scores for left bonds up to CHL (16, 32 or 64): each thread holds its
// branch's left-environment vector E_k[(lam, g)] in registers (read once per
// (g, e) instead of once per right index), and the staged block
// Ahat[(pd, e, g)] is read from shared memory in 16-byte vectors that every
// thread of a warp shares (broadcast), CHL rows zero-padded.
template <class CT, int CHL>
__global__ void __launch_bounds__(256) score_reg_kernel(int K, int d, int chl, int chr, int nG, int nE, int nPdr,
                                                        const double* E, const double* Ahat, const double* Ft,
                                                        const double* f, const double* w, const int32_t* lam_x,
                                                        const int32_t* u_x, const int32_t* pd_x, const int32_t* pr_x,
                                                        const int32_t* pdr_x, double* s) {
  constexpr int V = 16 / sizeof(CT);
  using Vec = typename std::conditional<sizeof(CT) == 4, float4, double2>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  CT* As = reinterpret_cast<CT*>(smraw);   // CHL x ldA
  const int ldA = (chr + V - 1) / V * V;
  const int x = blockIdx.x;
  CT acc[4] = {0, 0, 0, 0};
  for (int g = 0; g < nG; ++g)
    for (int e = 0; e < nE; ++e) {
      const double* A = Ahat + (((long long)pd_x[x] * nE + e) * nG + g) * chl * chr;
      __syncthreads();
      for (int i = threadIdx.x; i < CHL * ldA; i += blockDim.x) {
        const int al = i / ldA, ar = i % ldA;
        As[i] = (al < chl && ar < chr) ? CT(A[al * chr + ar]) : CT(0);
      }
      __syncthreads();
      const double* Eb = E + (long long)(lam_x[x] * nG + g) * chl * K;
      const double* Fb = Ft + (((long long)pr_x[x] * nE + e) * nPdr + pdr_x[x]) * chr * K;
      for (int j = 0; j < 4; ++j) {
        const int k = threadIdx.x + j * blockDim.x;
        if (k >= K) break;
        CT ev[CHL];
#pragma unroll
        for (int al = 0; al < CHL; ++al) ev[al] = al < chl ? CT(Eb[(long long)al * K + k]) : CT(0);
        CT a2 = 0;
        for (int ar0 = 0; ar0 < chr; ar0 += V) {
          CT t[V];
#pragma unroll
          for (int v = 0; v < V; ++v) t[v] = CT(0);
#pragma unroll
          for (int al = 0; al < CHL; ++al) {
            const Vec a = *reinterpret_cast<const Vec*>(As + al * ldA + ar0);
            const CT* av = reinterpret_cast<const CT*>(&a);
#pragma unroll
            for (int v = 0; v < V; ++v) t[v] = fma(ev[al], av[v], t[v]);
          }
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (ar0 + v < chr) a2 = fma(t[v], CT(Fb[(long long)(ar0 + v) * K + k]), a2);
        }
        acc[j] += a2;
      }
    }
  for (int j = 0; j < 4; ++j) {
    const int k = threadIdx.x + j * blockDim.x;
    if (k >= K) break;
    s[(long long)k * d + x] = f[(long long)u_x[x] * K + k] * w[x] * double(acc[j]);
  }
}

// log p of every candidate; invalid (score <= 0) -> key 0
__global__ void logp_kernel(int K, int d, const double* s, const double* logp_in, double* lp,
                            unsigned long long* key, int* clamps) {
  int k = blockIdx.x;
  __shared__ double red[32];
  double z = 0;
  int neg = 0;
  for (int x = threadIdx.x; x < d; x += blockDim.x) {
    double v = s[(long long)k * d + x];
    if (v > 0) z += v;
    if (v < 0) ++neg;
  }
  for (int o = 16; o > 0; o >>= 1) {
    z += __shfl_xor_sync(0xffffffffu, z, o);
    neg += __shfl_xor_sync(0xffffffffu, neg, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = z;
    if (neg) atomicAdd(clamps, neg);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  double Z = red[0];
  double base = logp_in[k];
  for (int x = threadIdx.x; x < d; x += blockDim.x) {
    double v = s[(long long)k * d + x];
    long long i = (long long)k * d + x;
    if (v > 0 && Z > 0) {
      double l = base + log(v / Z);
      lp[i] = l;
      key[i] = ord_key(l);
    } else {
      lp[i] = -INFINITY;
      key[i] = 0ull;
    }
  }
}

__global__ void merge1_kernel(int K, int d, int nX, const unsigned long long* key, const int32_t* pc,
                              const int32_t* xk, unsigned long long* best) {
  long long n = (long long)K * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!key[i]) continue;
    int k = int(i / d), x = int(i % d);
    atomicMax(best + (long long)pc[k] * nX + xk[x], key[i]);
  }
}
// every candidate within the tie tolerance of its group's maximum competes on configuration order
__global__ void merge2_kernel(int K, int d, int nX, const unsigned long long* key, const double* lp,
                              const int32_t* pc, const int32_t* prank, const int32_t* xk,
                              const unsigned long long* best, int* mn) {
  long long n = (long long)K * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!key[i]) continue;
    int k = int(i / d), x = int(i % d);
    long long slot = (long long)pc[k] * nX + xk[x];
    double top = key_to_double(best[slot]);
    if (lp[i] >= top - tie_tol(top)) atomicMin(mn + slot, prank[k] * d + x);
  }
}
// winners: key stays, losers: key -> 0 after recording them in `lost`
__global__ void merge3_kernel(int K, int d, int nX, unsigned long long* key, const int32_t* pc, const int32_t* prank,
                              const int32_t* xk, const int* mn, unsigned long long* lost) {
  long long n = (long long)K * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!key[i]) continue;
    int k = int(i / d), x = int(i % d);
    long long slot = (long long)pc[k] * nX + xk[x];
    if (mn[slot] != prank[k] * d + x) {
      atomicMax(lost, key[i]);
      key[i] = 0ull;
    }
  }
}

// histogram of digit `shift` among keys matching prefix on the higher bits
__global__ void hist_kernel(long long n, const unsigned long long* key, int shift, unsigned long long prefix,
                            unsigned long long pmask, unsigned int* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long k = key[i];
    if (!k || (k & pmask) != prefix) continue;
    atomicAdd(&h[(k >> shift) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, h[i]);
}

// above T + tol: selected; within T +- tol: tie class; other valid ones: p_d
__global__ void select_kernel(long long n, const unsigned long long* key, const double* lp, double T, double tol,
                              int* nsel, long long* sel, int* ntie, long long* tie, unsigned long long* lost,
                              int cap_sel, int cap_tie) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!key[i]) continue;
    double v = lp[i];
    if (v > T + tol) {
      int j = atomicAdd(nsel, 1);
      if (j < cap_sel) sel[j] = i;
    } else if (v >= T - tol) {
      int j = atomicAdd(ntie, 1);
      if (j < cap_tie) tie[j] = i;
    } else {
      atomicMax(lost, key[i]);
    }
  }
}

inline int nblk(long long n, int t = 256) {
  long long b = (n + t - 1) / t;
  return int(std::max(1ll, std::min(b, 148ll * 16)));
}

struct Step {
  sgtn_inst* h;
  int r, c, n, K;
  int32_t* dcfg = nullptr;   // [K][n] (n may be 0)
  int cfg_ld = 1;
  std::vector<double*> f;    // per column [nU][K]
  std::vector<double*> Ahat; // per column
  double* E = nullptr;       // left env [nBL(c)][chl(c)][K]
  double* Ft = nullptr;      // [nK(c)][chr(c)][K]
  double* s = nullptr;       // [K][d]
  const MPS* A = nullptr;
  std::vector<void*> owned;
  // optional caller-provided device arena: when set, alloc() carves from it
  // instead of calling cudaMalloc (256-byte aligned pieces)
  char* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  bool spill = false;        // arena exhausted: cudaMalloc the rest (the search grows its arena next step)
  size_t spilled = 0;
  template <class T>
  T* alloc(size_t n) {
    if (arena) {
      size_t b = ((n ? n : 1) * sizeof(T) + 255) / 256 * 256;
      if (arena_used + b <= arena_cap) {
        T* p = reinterpret_cast<T*>(arena + arena_used);
        arena_used += b;
        return p;
      }
      if (!spill) throw SgtnError(-1, "scratch arena exhausted");
      spilled += b;
    }
    void* p = pool_alloc((n ? n : 1) * sizeof(T));
    owned.push_back(p);
    return static_cast<T*>(p);
  }
  ~Step() {
    for (void* p : owned) pool_free(p);
  }
  const Column& col(int cc) const { return h->cols[r * h->M.C + cc]; }
};

// upper factors f[u][k] of column cc of row r for K branches (configs dcfg)
void launch_upper_f(sgtn_inst* h, int r, int cc, int K, const int32_t* dcfg, int cfg_ld, double* f) {
  const int C = h->M.C;
  const Column& K_ = h->cols[r * C + cc];
  const DSite* up = r > 0 ? &h->ds[(r - 1) * C + cc] : nullptr;
  const DSite& me = h->ds[r * C + cc];
  const int32_t *ul_pdr = nullptr, *ur_pdl = nullptr;
  const double *Bv = nullptr, *Bdr = nullptr, *Bdl = nullptr;
  int bv_nb = 1, bdr_nb = 1, bdl_nb = 1;
  const int32_t* up_pd = nullptr;
  if (r > 0) {
    up_pd = up->cls[DD];
    Bv = h->dB[size_t((r - 1) * C + cc) * 4 + 1];
    bv_nb = h->M.tab[size_t((r - 1) * C + cc) * 4 + 1].nB;
    if (cc - 1 >= 0) {
      ul_pdr = h->ds[(r - 1) * C + cc - 1].cls[DDR];
      Bdr = h->dB[size_t((r - 1) * C + cc - 1) * 4 + 2];
      bdr_nb = h->M.tab[size_t((r - 1) * C + cc - 1) * 4 + 2].nB;
    }
    if (cc + 1 < C) {
      ur_pdl = h->ds[(r - 1) * C + cc + 1].cls[DDL];
      Bdl = h->dB[size_t((r - 1) * C + cc + 1) * 4 + 3];
      bdl_nb = h->M.tab[size_t((r - 1) * C + cc + 1) * 4 + 3].nB;
    }
  }
  {
    KTimer kt("upper_f", h->st);
    upper_f_kernel<<<nblk((long long)K_.nU * K), 256, 0, h->st>>>(K, K_.nU, r, cc, C, dcfg, cfg_ld, up_pd, Bv, bv_nb,
                                                               me.U_u, ul_pdr, Bdr, bdr_nb, me.U_ul, ur_pdl, Bdl,
                                                               bdl_nb, me.U_ur, f);
  }
  ++g_count.launches;
}

// one step of the right environment: Fn [nBL][chl][K] from Ftl = Wk F [nK][chr][K]
// of column cc (unplaced: summed over its states with weights w and factors f),
// each branch's column normalised by its largest entry
void renv_step(sgtn_inst* h, int r, int cc, const double* Ahat, const double* Ftl, const double* f, int K, int chl,
               int chr, double* Fn) {
  const int C = h->M.C;
  const Column& K_ = h->cols[r * C + cc];
  cudaStream_t st = h->st;
  SGTN_CUDA(cudaMemsetAsync(Fn, 0, size_t(K_.nBL()) * chl * K * sizeof(double), st));
  SegGemm a;
  a.name = "renv";
  a.X = Ahat;
  a.p = chl;
  a.q = chr;
  a.xs_i = chr;
  a.xs_k = 1;
  a.xrs = (long long)chl * chr;
  a.Y = Ftl;
  a.s = K;
  a.ys_k = K;
  a.ys_j = 1;
  a.yrs = (long long)chr * K;
  a.O = Fn;
  a.os_i = K;
  a.os_j = 1;
  a.ors = (long long)chl * K;
  a.seg_ptr = K_.renv.seg_ptr;
  a.vseg_ptr = K_.renv.vseg_ptr;
  a.vfirst = K_.renv.vfirst;
  a.nvseg = K_.renv.nvseg;
  a.seg_or = K_.renv.seg_or;
  a.seg_oc = K_.renv.seg_oc;
  a.xr = K_.renv.xr;
  a.xc = K_.renv.xc;
  a.yr = K_.renv.yr;
  a.yc = K_.renv.yc;
  a.cidx = K_.renv.cidx;
  a.csrow = K_.renv.csrow;
  a.coef = h->ds[r * C + cc].w;
  a.cs = f;
  a.cs_ld = K;
  a.nseg = K_.renv.nseg;
  a.nterm = K_.renv.nterm;
  seg_gemm(a, st);
  colnorm_kernel<<<K, 256, 0, st>>>(Fn, (long long)K_.nBL() * chl, K);
  ++g_count.launches;
}

// new left environment Eout [nBR(cc)][chr][Kout] after placing column cc:
// branch kk extends branch par[kk] of Ein (Kin branches) with state xs[kk]
void lenv_step(sgtn_inst* h, int r, int cc, const double* Ahat, const double* Ein, int Kin, int Kout,
               const int32_t* par, const int32_t* xs, int chl, int chr, double* Eout) {
  const int C = h->M.C;
  const Column& K_ = h->cols[r * C + cc];
  const DSite& D = h->ds[r * C + cc];
  size_t smem = size_t(K_.nE) * chr * sizeof(double);
  {
    KTimer kt("lenv", h->st);
    lenv_kernel<<<Kout, 128, smem, h->st>>>(Kin, Kout, par, xs, Ein, chl, chr, K_.nG, K_.nE, K_.nPdr, K_.nLR, K_.nGR,
                                          Ahat, D.lam_x, D.cls[DD], D.cls[DR_], D.cls[DDR], K_.l_pl, K_.l_pdl,
                                          h->dB[size_t(r * C + cc) * 4 + 0], K_.bh_nb,
                                          h->dB[size_t(r * C + cc) * 4 + 2], K_.bdr_nb, Eout);
  }
  ++g_count.launches;
}

// scores S.s[k][x] of column S.c from S.E, S.Ahat[c], S.f[c] and Ft = Wk F
void compute_scores(Step& S, const double* Ft) {
  sgtn_inst* h = S.h;
  cudaStream_t st = h->st;
  const int r = S.r, c = S.c, K = S.K;
  const Column& Kc = S.col(c);
  const int chl = S.A->bond[c], chr = S.A->bond[c + 1];
  const DSite& D = h->ds[r * h->M.C + c];
  S.s = S.alloc<double>(size_t(K) * D.d);
  int thr = std::min(256, std::max(32, ((K + 3) / 4 + 31) / 32 * 32));
  if (K > 4 * thr) throw SgtnError(-1, "beam too large for the score kernel");
  double sc_fl = 2.0 * K * D.d * (double)Kc.nG * Kc.nE * chl * (chr + 1);
  // left bonds up to 64 (every chi <= 64): the register form
  auto reg = [&](auto ct, auto chlmax) {
    using CT = decltype(ct);
    constexpr int CHL = decltype(chlmax)::value;
    constexpr int V = 16 / sizeof(CT);
    const size_t smem = size_t(CHL) * ((chr + V - 1) / V * V) * sizeof(CT);
    score_reg_kernel<CT, CHL><<<D.d, thr, smem, st>>>(K, D.d, chl, chr, Kc.nG, Kc.nE, Kc.nPdr, S.E, S.Ahat[c], Ft,
                                                      S.f[c], D.w, D.lam_x, D.u_x, D.cls[DD], D.cls[DR_], D.cls[DDR],
                                                      S.s);
  };
  using I16 = std::integral_constant<int, 16>;
  using I32 = std::integral_constant<int, 32>;
  using I64 = std::integral_constant<int, 64>;
  if (g_compute_f32) {
    KTimer tsc("score_f32", st, sc_fl);
    if (chl <= 16) reg(float(), I16());
    else if (chl <= 32) reg(float(), I32());
    else if (chl <= 64) reg(float(), I64());
    else
      score_kernel<float><<<D.d, thr, size_t(chl) * chr * sizeof(float), st>>>(
          K, D.d, chl, chr, Kc.nG, Kc.nE, Kc.nPdr, S.E, S.Ahat[c], Ft, S.f[c], D.w, D.lam_x, D.u_x, D.cls[DD],
          D.cls[DR_], D.cls[DDR], S.s);
  } else {
    KTimer tsc("score_f64", st, sc_fl);
    if (chl <= 16) reg(double(), I16());
    else if (chl <= 32) reg(double(), I32());
    else if (chl <= 64) reg(double(), I64());
    else
      score_kernel<double><<<D.d, thr, size_t(chl) * chr * sizeof(double), st>>>(
          K, D.d, chl, chr, Kc.nG, Kc.nE, Kc.nPdr, S.E, S.Ahat[c], Ft, S.f[c], D.w, D.lam_x, D.u_x, D.cls[DD],
          D.cls[DR_], D.cls[DDR], S.s);
  }
  ++g_count.launches;
}

// everything up to the unnormalised scores s[k][x], from scratch (stateless
// entry points: conditionals, branch_step)
void prepare_scores(Step& S, const int32_t* hcfg) {
  sgtn_inst* h = S.h;
  cudaStream_t st = h->st;
  const int C = h->M.C;
  const int r = S.r, c = S.c, K = S.K;
  if (!h->boundary_ok) throw SgtnError(-2, "contract_boundary must run first");
  S.A = &h->psi[r];
  S.cfg_ld = std::max(S.n, 1);
  S.dcfg = S.alloc<int32_t>(size_t(K) * S.cfg_ld);
  if (S.n > 0)
    SGTN_CUDA(cudaMemcpyAsync(S.dcfg, hcfg, size_t(K) * S.n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  // projected MPS of psi_r, every column
  S.Ahat.assign(C, nullptr);
  for (int cc = 0; cc < C; ++cc) {
    const Column& K_ = S.col(cc);
    long long blk = (long long)S.A->bond[cc] * S.A->bond[cc + 1];
    S.Ahat[cc] = S.alloc<double>(size_t(K_.nA() * blk));
    gemm(K_.Wa, false, K_.nSig, S.A->t[cc], false, blk, S.Ahat[cc], blk, K_.nA(), int(blk), K_.nSig, 1.0, 0, st);
  }
  // upper factors
  S.f.assign(C, nullptr);
  for (int cc = 0; cc < C; ++cc) {
    S.f[cc] = S.alloc<double>(size_t(S.col(cc).nU) * K);
    launch_upper_f(h, r, cc, K, S.dcfg, S.cfg_ld, S.f[cc]);
  }
  // left environment at column c
  {
    S.E = S.alloc<double>(K);
    fill(S.E, K, 1.0, st);
    int32_t* par = S.alloc<int32_t>(K);
    int32_t* xs = S.alloc<int32_t>(K);
    SGTN_CUDA(cudaMemcpyAsync(par, h->iota, K * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    for (int cc = 0; cc < c; ++cc) {
      const Column& K_ = S.col(cc);
      std::vector<int32_t> hx(K);
      for (int k = 0; k < K; ++k) hx[k] = hcfg[(long long)k * S.n + r * C + cc];
      SGTN_CUDA(cudaMemcpyAsync(xs, hx.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      int chl = S.A->bond[cc], chr = S.A->bond[cc + 1];
      double* En = S.alloc<double>(size_t(K_.nBR()) * chr * K);
      lenv_step(h, r, cc, S.Ahat[cc], S.E, K, K, par, xs, chl, chr, En);
      S.E = En;
      h->sync();  // xs is reused
    }
  }
  // right environment at bond (c, c+1)
  double* F = S.alloc<double>(K);
  fill(F, K, 1.0, st);
  for (int cc = C - 1; cc > c; --cc) {
    const Column& K_ = S.col(cc);
    int chl = S.A->bond[cc], chr = S.A->bond[cc + 1];
    double* Ftl = S.alloc<double>(size_t(K_.nK()) * chr * K);
    gemm(K_.Wk, false, K_.nBR(), F, false, (long long)chr * K, Ftl, (long long)chr * K, K_.nK(), chr * K, K_.nBR(), 1.0,
         0, st);
    double* Fn = S.alloc<double>(size_t(K_.nBL()) * chl * K);
    renv_step(h, r, cc, S.Ahat[cc], Ftl, S.f[cc], K, chl, chr, Fn);
    F = Fn;
  }
  const Column& Kc = S.col(c);
  int chr = S.A->bond[c + 1];
  S.Ft = S.alloc<double>(size_t(Kc.nK()) * chr * K);
  gemm(Kc.Wk, false, Kc.nBR(), F, false, (long long)chr * K, S.Ft, (long long)chr * K, Kc.nK(), chr * K, Kc.nBR(), 1.0, 0,
       st);
  compute_scores(S, S.Ft);
  h->check();
}

void check_configs(sgtn_inst* h, int step, int count, const int32_t* cfg) {
  const int RC = h->M.R * h->M.C;
  if (step < 0 || step >= RC) throw SgtnError(-1, "step out of range");
  if (count <= 0) throw SgtnError(-1, "count must be positive");
  // the score kernel holds at most SGTN_MAX_BEAM branches per CTA, and the
  // initial parent list is a prefix of the handle's iota table
  if (count > SGTN_MAX_BEAM || count > h->iota_n)
    throw SgtnError(-1, "count " + std::to_string(count) + " exceeds SGTN_MAX_BEAM (" + std::to_string(SGTN_MAX_BEAM) +
                            ")");
  if (step > 0 && !cfg) throw SgtnError(-1, "configs is NULL");
  for (long long k = 0; k < count; ++k)
    for (int p = 0; p < step; ++p) {
      int x = cfg[k * step + p];
      if (x < 0 || x >= h->M.sites[p].d) throw SgtnError(-1, "state index out of range");
    }
}

}  // namespace

void conditionals(sgtn_inst* h, int step, int count, const int32_t* configs, double* out_p) {
  check_configs(h, step, count, configs);
  if (!out_p) throw SgtnError(-1, "out_p is NULL");
  Step S;
  S.h = h;
  S.n = step;
  S.r = step / h->M.C;
  S.c = step % h->M.C;
  S.K = count;
  prepare_scores(S, configs);
  int d = h->M.sites[step].d;
  std::vector<double> s(size_t(count) * d);
  SGTN_CUDA(cudaMemcpyAsync(s.data(), S.s, s.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  for (int k = 0; k < count; ++k) {
    double z = 0;
    for (int x = 0; x < d; ++x) z += std::max(0.0, s[size_t(k) * d + x]);
    for (int x = 0; x < d; ++x) out_p[size_t(k) * d + x] = z > 0 ? std::max(0.0, s[size_t(k) * d + x]) / z : 0.0;
  }
}

// Device bytes prepare_scores takes from an arena (same pieces, same rounding).
size_t scores_scratch_bytes(sgtn_inst* h, int step, int K) {
  const int C = h->M.C, r = step / C, c = step % C;
  if (!h->boundary_ok) throw SgtnError(-2, "contract_boundary must run first");
  const MPS& A = h->psi[r];
  auto rnd = [](size_t b) { return ((b ? b : 1) + 255) / 256 * 256; };
  size_t tot = rnd(size_t(K) * std::max(step, 1) * sizeof(int32_t));
  for (int cc = 0; cc < C; ++cc) {
    const Column& K_ = h->cols[r * C + cc];
    tot += rnd(size_t(K_.nA()) * A.bond[cc] * A.bond[cc + 1] * sizeof(double));
    tot += rnd(size_t(K_.nU) * K * sizeof(double));
  }
  tot += rnd(size_t(K) * sizeof(double)) + 2 * rnd(size_t(K) * sizeof(int32_t));
  for (int cc = 0; cc < c; ++cc)
    tot += rnd(size_t(h->cols[r * C + cc].nBR()) * A.bond[cc + 1] * K * sizeof(double));
  tot += rnd(size_t(K) * sizeof(double));
  for (int cc = C - 1; cc > c; --cc) {
    const Column& K_ = h->cols[r * C + cc];
    tot += rnd(size_t(K_.nK()) * A.bond[cc + 1] * K * sizeof(double));
    tot += rnd(size_t(K_.nBL()) * A.bond[cc] * K * sizeof(double));
  }
  tot += rnd(size_t(h->cols[r * C + c].nK()) * A.bond[c + 1] * K * sizeof(double));
  tot += rnd(size_t(K) * h->M.sites[step].d * sizeof(double));
  return tot;
}

// Conditional marginals with every device temporary carved from `arena`
// (no device allocation); writes straight into the caller's out_p.
void conditionals_arena(sgtn_inst* h, int step, int count, const int32_t* configs, double* out_p, void* arena,
                        size_t cap) {
  check_configs(h, step, count, configs);
  if (!out_p) throw SgtnError(-1, "out_p is NULL");
  size_t need = scores_scratch_bytes(h, step, count);
  if (need > cap)
    throw SgtnError(-1, "this call needs " + std::to_string(need) + " bytes of device scratch; the static buffer holds " +
                            std::to_string(cap) + " (reduce count or use sgtn_conditionals)");
  Step S;
  S.h = h;
  S.n = step;
  S.r = step / h->M.C;
  S.c = step % h->M.C;
  S.K = count;
  S.arena = static_cast<char*>(arena);
  S.arena_cap = cap;
  struct NoAlloc {
    bool saved = g_no_alloc;
    NoAlloc() { g_no_alloc = true; }
    ~NoAlloc() { g_no_alloc = saved; }
  } no_alloc;
  prepare_scores(S, configs);
  int d = h->M.sites[step].d;
  SGTN_CUDA(cudaMemcpyAsync(out_p, S.s, size_t(count) * d * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  h->sync();
  for (int k = 0; k < count; ++k) {
    double* row = out_p + size_t(k) * d;
    double z = 0;
    for (int x = 0; x < d; ++x) z += std::max(0.0, row[x]);
    for (int x = 0; x < d; ++x) row[x] = z > 0 ? std::max(0.0, row[x]) / z : 0.0;
  }
}

// Steps 3-5 from the scores S.s of the K = S.K branches: log p, merge, top-M.
// out_parent (optional) receives the branch index of every survivor.
// One step's merges seen from the host, for the droplet bookkeeping of
// Fig. 4: every valid candidate that was merged away while its group's winner
// survived the top-M cut, with that winner's position in the kept list.
struct MergeLosers {
  std::vector<long long> cand;   // candidate index k * d + x
  std::vector<int> winner;
};

void select_step(Step& S, int step, int M, const int32_t* in_configs, const double* in_logp, int32_t* out_configs,
                 double* out_logp, int32_t* out_count, double* io_pd, int32_t* out_parent,
                 MergeLosers* losers = nullptr) {
  sgtn_inst* h = S.h;
  cudaStream_t st = h->st;
  const int C = h->M.C;
  const int K = S.K;
  const HSite& site = h->M.sites[step];
  const int d = site.d;
  const long long ncand = (long long)K * d;
  double* dlp_in = S.alloc<double>(K);
  SGTN_CUDA(cudaMemcpyAsync(dlp_in, in_logp, K * sizeof(double), cudaMemcpyHostToDevice, st));
  double* lp = S.alloc<double>(ncand);
  unsigned long long* key = S.alloc<unsigned long long>(ncand);
  int* clamps = S.alloc<int>(1);
  SGTN_CUDA(cudaMemsetAsync(clamps, 0, sizeof(int), st));
  {
    KTimer kt("logp", h->st);
    logp_kernel<<<K, 256, 0, st>>>(K, d, S.s, dlp_in, lp, key, clamps);
  }
  g_count.evals += ncand; ++g_count.launches;
  // parent classes from the boundary pairs (p, dir) with p < step < l (Eq. 7):
  // pc[k] = smallest branch with the same vector of boundary classes, prank[k]
  // = position of branch k's configuration in lexicographic order (ties by
  // index).  Both come from two sorts on the host, which holds the configs.
  std::vector<int32_t> psite;
  std::vector<const int32_t*> hcls;
  for (int p = 0; p < step; ++p) {
    const HSite& P = h->M.sites[p];
    for (int dd = 0; dd < 8; ++dd) {
      int rr = P.r + kDr[dd], cc = P.c + kDc[dd];
      if (rr < 0 || rr >= h->M.R || cc < 0 || cc >= C) continue;
      int l = rr * C + cc;
      if (l > step && !P.coupled[dd].empty()) {
        psite.push_back(p);
        hcls.push_back(P.proj[dd].of_state.data());
      }
    }
  }
  const int npairs = int(psite.size());
  std::vector<int32_t> hpc(K), hprank(K), order(K);
  {
    auto cfgp = [&](int k) { return in_configs + (long long)k * step; };
    auto same_classes = [&](int a, int b) {
      const int32_t *ca = cfgp(a), *cb = cfgp(b);
      for (int j = 0; j < npairs; ++j)
        if (hcls[j][ca[psite[j]]] != hcls[j][cb[psite[j]]]) return false;
      return true;
    };
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      const int32_t *ca = cfgp(a), *cb = cfgp(b);
      for (int j = 0; j < npairs; ++j) {
        const int32_t x = hcls[j][ca[psite[j]]], y = hcls[j][cb[psite[j]]];
        if (x != y) return x < y;
      }
      return a < b;
    });
    for (int i = 0; i < K; ++i) {
      const int k = order[i];
      hpc[k] = (i > 0 && same_classes(k, order[i - 1])) ? hpc[order[i - 1]] : k;
    }
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      const int32_t *ca = cfgp(a), *cb = cfgp(b);
      for (int j = 0; j < step; ++j)
        if (ca[j] != cb[j]) return ca[j] < cb[j];
      return a < b;
    });
    for (int i = 0; i < K; ++i) hprank[order[i]] = i;
  }
  int32_t* pc = S.alloc<int32_t>(K);
  int32_t* prank = S.alloc<int32_t>(K);
  SGTN_CUDA(cudaMemcpyAsync(pc, hpc.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SGTN_CUDA(cudaMemcpyAsync(prank, hprank.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  const int nX = site.Xk.n;
  long long nslot = (long long)K * nX;
  unsigned long long* best = S.alloc<unsigned long long>(nslot);
  int* mn = S.alloc<int>(nslot);
  SGTN_CUDA(cudaMemsetAsync(best, 0, nslot * sizeof(unsigned long long), st));
  SGTN_CUDA(cudaMemsetAsync(mn, 0x7f, nslot * sizeof(int), st));
  unsigned long long* lost = S.alloc<unsigned long long>(1);
  SGTN_CUDA(cudaMemsetAsync(lost, 0, sizeof(unsigned long long), st));
  {
    KTimer kt("merge1", h->st);
    merge1_kernel<<<nblk(ncand), 256, 0, st>>>(K, d, nX, key, pc, h->ds[step].xk_x, best);
  } ++g_count.launches;
  {
    KTimer kt("merge2", h->st);
    merge2_kernel<<<nblk(ncand), 256, 0, st>>>(K, d, nX, key, lp, pc, prank, h->ds[step].xk_x, best, mn);
  } ++g_count.launches;
  {
    KTimer kt("merge3", h->st);
    merge3_kernel<<<nblk(ncand), 256, 0, st>>>(K, d, nX, key, pc, prank, h->ds[step].xk_x, mn, lost);
  } ++g_count.launches;
  // radix select of the M-th largest key
  unsigned int* hist = S.alloc<unsigned int>(256);
  unsigned long long prefix = 0, pmask = 0;
  long long need = M;
  long long total_valid = 0;
  {
    // count valid survivors first (histogram of the top digit with empty prefix)
    SGTN_CUDA(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st));
    hist_kernel<<<nblk(ncand), 256, 0, st>>>(ncand, key, 56, 0ull, 0ull, hist); ++g_count.launches;
    std::vector<unsigned int> hh(256);
    SGTN_CUDA(cudaMemcpyAsync(hh.data(), hist, 256 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    h->sync();
    for (auto v : hh) total_valid += v;
    if (total_valid == 0) throw SgtnError(-4, "no candidate with a positive score");
    double T = -INFINITY, tol = 0.0;
    if (total_valid > M) {
      for (int shift = 56; shift >= 0; shift -= 8) {
        if (shift != 56) {
          SGTN_CUDA(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st));
          hist_kernel<<<nblk(ncand), 256, 0, st>>>(ncand, key, shift, prefix, pmask, hist); ++g_count.launches;
          SGTN_CUDA(cudaMemcpyAsync(hh.data(), hist, 256 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
          h->sync();
        }
        int b = 255;
        for (; b >= 0; --b) {
          if ((long long)hh[b] >= need) break;
          need -= hh[b];
        }
        prefix |= (unsigned long long)b << shift;
        pmask |= 255ull << shift;
      }
      T = key_to_double(prefix);   // the M-th largest log p
      tol = tie_tol(T);
    }
    int* nsel = S.alloc<int>(2);
    SGTN_CUDA(cudaMemsetAsync(nsel, 0, 2 * sizeof(int), st));
    // a tie class may be as large as the candidate set (degenerate instances)
    int cap_sel = M + 1, cap_tie = int(std::min<long long>(ncand, INT_MAX));
    long long* sel = S.alloc<long long>(cap_sel);
    long long* tie = S.alloc<long long>(cap_tie);
    {
      KTimer kt("select", h->st);
      select_kernel<<<nblk(ncand), 256, 0, st>>>(ncand, key, lp, T, tol, nsel, sel, nsel + 1, tie, lost, cap_sel,
                                               cap_tie);
    } ++g_count.launches;
    int hn[2];
    SGTN_CUDA(cudaMemcpyAsync(hn, nsel, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    h->sync();
    int n_above = hn[0], n_tie = hn[1];
    if (n_above > M || n_tie > cap_tie) throw SgtnError(-4, "too many tied candidates at the top-M cut");
    std::vector<long long> hsel(n_above), htie(n_tie);
    if (n_above) SGTN_CUDA(cudaMemcpyAsync(hsel.data(), sel, n_above * sizeof(long long), cudaMemcpyDeviceToHost, st));
    if (n_tie) SGTN_CUDA(cudaMemcpyAsync(htie.data(), tie, n_tie * sizeof(long long), cudaMemcpyDeviceToHost, st));
    std::vector<double> hlp(ncand);
    SGTN_CUDA(cudaMemcpyAsync(hlp.data(), lp, ncand * sizeof(double), cudaMemcpyDeviceToHost, st));
    unsigned long long hlost = 0;
    SGTN_CUDA(cudaMemcpyAsync(&hlost, lost, sizeof(hlost), cudaMemcpyDeviceToHost, st));
    h->sync();
    auto cfg_order = [&](long long a) { return (long long)hprank[a / d] * d + a % d; };
    // the tie class is filled in configuration order
    std::sort(htie.begin(), htie.end(), [&](long long a, long long b) { return cfg_order(a) < cfg_order(b); });
    std::vector<long long> keep = hsel;
    for (int i = 0; i < n_tie; ++i) {
      if ((long long)keep.size() < M)
        keep.push_back(htie[i]);
      else
        hlost = std::max(hlost, ord_key(hlp[htie[i]]));
    }
    std::sort(keep.begin(), keep.end(), [&](long long a, long long b) {
      if (hlp[a] != hlp[b]) return hlp[a] > hlp[b];
      return cfg_order(a) < cfg_order(b);
    });
    int outc = int(keep.size());
    for (int i = 0; i < outc; ++i) {
      long long ci = keep[i];
      int k = int(ci / d), x = int(ci % d);
      for (int p = 0; p < step; ++p) out_configs[(long long)i * (step + 1) + p] = in_configs[(long long)k * step + p];
      out_configs[(long long)i * (step + 1) + step] = x;
      out_logp[i] = hlp[ci];
      if (out_parent) out_parent[i] = k;
    }
    *out_count = outc;
    if (hlost) *io_pd = std::max(*io_pd, key_to_double(hlost));
    if (losers) {
      // merge groups are (parent class, class of x toward the unplaced sites)
      const std::vector<int32_t>& xkc = site.Xk.of_state;
      std::unordered_map<long long, int> win_of;
      for (int i = 0; i < outc; ++i) {
        const long long ci = keep[i];
        win_of[(long long)hpc[ci / d] * nX + xkc[ci % d]] = i;
      }
      for (long long ci = 0; ci < ncand; ++ci) {
        if (!(hlp[ci] > -INFINITY)) continue;
        auto it = win_of.find((long long)hpc[ci / d] * nX + xkc[ci % d]);
        if (it == win_of.end() || keep[it->second] == ci) continue;
        losers->cand.push_back(ci);
        losers->winner.push_back(it->second);
      }
    }
  }
  h->check();
  (void)C;
}

void branch_step(sgtn_inst* h, int step, int M, int in_count, const int32_t* in_configs, const double* in_logp,
                 int32_t* out_configs, double* out_logp, int32_t* out_count, double* io_pd) {
  check_configs(h, step, in_count, in_configs);
  if (M <= 0 || !in_logp || !out_configs || !out_logp || !out_count || !io_pd) throw SgtnError(-1, "bad argument");
  const int C = h->M.C;
  Step S;
  S.h = h;
  S.n = step;
  S.r = step / C;
  S.c = step % C;
  S.K = in_count;
  prepare_scores(S, in_configs);
  select_step(S, step, M, in_configs, in_logp, out_configs, out_logp, out_count, io_pd, nullptr);
}

namespace {
// Host-side droplet bookkeeping (Fig. 4).  A main branch keeps its parent's
// droplets, then takes its merged-away candidates in order of (dE,
// configuration): each one's own droplet (the spins where it differs from the
// main branch, with the exact energy change) and its parent's droplets
// carried over (F xor F', dE + dE').  A droplet is kept if dE <= max_dE, its
// spins are connected in the interaction graph (J != 0), and it replaces
// every kept droplet within min_hamming flips only if its dE is lower than
// all of theirs.  Energies are exact int64 numerators: the energy of the
// placed clusters changes by E_x plus the compressed couplings to the placed
// neighbours (Eq. 2), and spins coupled to unplaced clusters are equal across
// a merge group, so dE holds for every completion.
struct DropletBook {
  sgtn_inst* h;
  DropletOpts opt;
  std::vector<std::vector<int32_t>> adj;
  std::vector<std::vector<Drop>> drops{std::vector<Drop>()};
  std::vector<long long> ep{0};          // energy of the placed clusters, per beam entry
  std::vector<char> mark;

  DropletBook(sgtn_inst* hh, const DropletOpts& o) : h(hh), opt(o) {
    const Model& M = h->M;
    adj.assign(M.N, {});
    for (size_t e = 0; e < M.ei.size(); ++e)
      if (M.jn[e] != 0) {
        adj[M.ei[e]].push_back(M.ej[e]);
        adj[M.ej[e]].push_back(M.ei[e]);
      }
    mark.assign(M.N, 0);
  }
  // energy added by placing state x at `step` after the parent configuration pc
  long long inc(int step, const int32_t* pc, int x) const {
    const Model& M = h->M;
    const int C = M.C, r = step / C, c = step % C;
    const HSite& S = M.sites[step];
    long long e = S.E[x];
    auto add = [&](int q, int slot, Dir dq, Dir ds) {
      const HTable& T = M.tab[size_t(q) * 4 + slot];
      const int a = M.sites[q].proj[dq].of_state[pc[q]], b = S.proj[ds].of_state[x];
      e += T.E[size_t(a) * T.nB + b];
    };
    if (c > 0) add(step - 1, 0, DR_, DL_);
    if (r > 0) add(step - C, 1, DD, DU);
    if (r > 0 && c > 0) add(step - C - 1, 2, DDR, DUL);
    if (r > 0 && c + 1 < C) add(step - C + 1, 3, DDL, DUR);
    return e;
  }
  bool connected(const std::vector<int32_t>& F) {
    if (F.empty()) return false;
    for (int v : F) mark[v] = 1;
    std::vector<int32_t> todo{F[0]};
    mark[F[0]] = 2;
    size_t seen = 1;
    while (!todo.empty()) {
      const int u = todo.back();
      todo.pop_back();
      for (int v : adj[u])
        if (mark[v] == 1) {
          mark[v] = 2;
          ++seen;
          todo.push_back(v);
        }
    }
    for (int v : F) mark[v] = 0;
    return seen == F.size();
  }
  static std::vector<int32_t> symdiff(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    std::vector<int32_t> o;
    std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(o));
    return o;
  }
  static size_t hamming(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    size_t i = 0, j = 0, n = 0;
    while (i < a.size() && j < b.size()) {
      if (a[i] == b[j]) ++i, ++j;
      else if (a[i] < b[j]) ++i, ++n;
      else ++j, ++n;
    }
    return n + (a.size() - i) + (b.size() - j);
  }
  void insert(std::vector<Drop>& lst, Drop&& cand) {
    if (cand.dE > opt.max_dE || !connected(cand.flips)) return;
    std::vector<size_t> clash;
    long long lo = LLONG_MAX;
    for (size_t i = 0; i < lst.size(); ++i)
      if (hamming(lst[i].flips, cand.flips) <= size_t(opt.min_hamming)) {
        clash.push_back(i);
        lo = std::min(lo, lst[i].dE);
      }
    if (clash.empty()) {
      lst.push_back(std::move(cand));
    } else if (cand.dE < lo) {
      std::vector<Drop> keep;
      size_t q = 0;
      for (size_t i = 0; i < lst.size(); ++i) {
        if (q < clash.size() && clash[q] == i) {
          ++q;
          continue;
        }
        keep.push_back(std::move(lst[i]));
      }
      keep.push_back(std::move(cand));
      lst.swap(keep);
    }
  }
  // spins where configuration (row a of A + xa) and (row b of B + xb) differ
  std::vector<int32_t> flips(int step, const int32_t* pa, int xa, const int32_t* pb, int xb) const {
    const Model& M = h->M;
    std::vector<int32_t> F;
    for (int p = 0; p <= step; ++p) {
      const int sa = p < step ? pa[p] : xa, sb = p < step ? pb[p] : xb;
      if (sa == sb) continue;
      const HSite& P = M.sites[p];
      const int64_t z = P.states[sa] ^ P.states[sb];
      for (size_t j = 0; j < P.spins.size(); ++j)
        if ((z >> j) & 1) F.push_back(P.spins[j]);
    }
    std::sort(F.begin(), F.end());
    return F;
  }
  // after select_step: cfg (stride step) the old beam, ncfg (stride step+1) the kept one
  void step(int step, const std::vector<int32_t>& cfg, const std::vector<int32_t>& ncfg, int oc,
            const std::vector<int32_t>& par, const MergeLosers& ml) {
    const int d = h->M.sites[step].d, w1 = step + 1;
    auto prow = [&](int k) { return cfg.data() + (size_t)k * step; };
    std::vector<long long> nep(oc);
    for (int i = 0; i < oc; ++i) nep[i] = ep[par[i]] + inc(step, prow(par[i]), ncfg[(size_t)i * w1 + step]);
    std::vector<std::vector<std::pair<long long, long long>>> byw(oc);
    for (size_t j = 0; j < ml.cand.size(); ++j) {
      const long long ci = ml.cand[j];
      const int k = int(ci / d), x = int(ci % d), w = ml.winner[j];
      byw[w].push_back({ep[k] + inc(step, prow(k), x) - nep[w], ci});
    }
    std::vector<std::vector<Drop>> nd(oc);
    for (int i = 0; i < oc; ++i) {
      std::vector<Drop> lst = drops[par[i]];
      auto& L = byw[i];
      std::sort(L.begin(), L.end(), [&](const std::pair<long long, long long>& a, const std::pair<long long, long long>& b) {
        if (a.first != b.first) return a.first < b.first;
        const int ka = int(a.second / d), kb = int(b.second / d);
        const int32_t *ra = prow(ka), *rb = prow(kb);
        for (int p = 0; p < step; ++p)
          if (ra[p] != rb[p]) return ra[p] < rb[p];
        return a.second % d < b.second % d;
      });
      const int32_t* wrow = prow(par[i]);
      const int wx = ncfg[(size_t)i * w1 + step];
      for (const auto& lc : L) {
        const long long dE = lc.first;
        const int k = int(lc.second / d), x = int(lc.second % d);
        const std::vector<Drop>& pl = drops[k];
        long long lo = dE;
        for (const Drop& q : pl) lo = std::min(lo, dE + q.dE);
        if (lo > opt.max_dE) continue;   // nothing from this candidate fits the window
        const std::vector<int32_t> F = flips(step, wrow, wx, prow(k), x);
        insert(lst, Drop{dE, F});
        for (const Drop& q : pl) insert(lst, Drop{dE + q.dE, symdiff(F, q.flips)});
      }
      nd[i] = std::move(lst);
    }
    drops.swap(nd);
    ep.swap(nep);
  }
};
}  // namespace

void search(sgtn_inst* h, int M, int n_out, int8_t* out_spins, int64_t* out_energy, double* out_logp, double* out_pd,
            int32_t* out_count, const DropletOpts* dopt, std::vector<Drop>* dout) {
  if (!h->boundary_ok) throw SgtnError(-2, "contract_boundary must run first");
  if (M <= 0 || n_out <= 0 || !out_spins || !out_energy || !out_logp || !out_pd || !out_count)
    throw SgtnError(-1, "bad argument");
  cudaStream_t st = h->st;
  const int C = h->M.C, RC = h->M.R * h->M.C;
  {
    // with large clusters the boundary's workspaces (named buffers and cached
    // pool blocks, kept for the next contraction) can hold most of the device
    // memory: when less than a quarter is free they are released here (the
    // boundary MPSs stay); later calls allocate again what they need
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr < tot / 4) {
      h->sync();
      pool_trim(st);
      h->ws.release();
    }
  }
  std::vector<int32_t> cfg(1, 0), ncfg;
  std::vector<double> lp(1, 0.0), nlp;
  int count = 1;
  double pd = -INFINITY;
  // Row cache: at the first column of row r everything that depends only on
  // psi_r and on each branch's fixed row r-1 -- the projected MPS Ahat, the
  // upper factors f and the right environments Ft = Wk F at every bond -- is
  // computed once for the branches alive then (K0 of them).  A later branch
  // inherits row r-1 from its ancestor anc[k] among those, so its f and Ft
  // are gathered, not recomputed; the left environment grows by one column
  // per step from the parent's.  Same values as the stateless branch step.
  std::vector<double*> Ahat(C, nullptr), fr(C, nullptr), Ft(C, nullptr);
  std::vector<int32_t> anc, par;
  int K0 = 0, Kprev = 0;
  double* E = nullptr;
  int ebuf = 0;
  size_t cap = size_t(64) << 20;   // per-step scratch; grows after a step that needed more
  std::unique_ptr<DropletBook> book;
  if (dopt) book.reset(new DropletBook(h, *dopt));
  for (int step = 0; step < RC; ++step) {
    const int r = step / C, c = step % C, K = count;
    // M may exceed SGTN_MAX_BEAM (a cap the bounding never reaches, e.g. to
    // disable the top-M cut on a narrow lattice); the live beam may not
    if (K > SGTN_MAX_BEAM)
      throw SgtnError(-1, "the beam grew to " + std::to_string(K) + " branches, above SGTN_MAX_BEAM (" +
                              std::to_string(SGTN_MAX_BEAM) + "): lower M");
    Step S;
    S.h = h;
    S.n = step;
    S.r = r;
    S.c = c;
    S.K = K;
    S.A = &h->psi[r];
    S.arena = h->ws.get<char>("search_arena", cap);
    S.arena_cap = cap;
    S.spill = true;
    S.cfg_ld = std::max(step, 1);
    S.dcfg = S.alloc<int32_t>(size_t(K) * S.cfg_ld);
    if (step > 0)
      SGTN_CUDA(cudaMemcpyAsync(S.dcfg, cfg.data(), size_t(K) * step * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (c == 0) {
      K0 = K;
      for (int cc = 0; cc < C; ++cc) {
        const Column& K_ = S.col(cc);
        const long long blk = (long long)S.A->bond[cc] * S.A->bond[cc + 1];
        Ahat[cc] = h->ws.get<double>("srch_A" + std::to_string(cc), size_t(K_.nA() * blk));
        gemm(K_.Wa, false, K_.nSig, S.A->t[cc], false, blk, Ahat[cc], blk, K_.nA(), int(blk), K_.nSig, 1.0, 0, st);
        fr[cc] = h->ws.get<double>("srch_f" + std::to_string(cc), size_t(K_.nU) * K0);
        launch_upper_f(h, r, cc, K0, S.dcfg, S.cfg_ld, fr[cc]);
      }
      double* F = h->ws.get<double>("srch_F1", size_t(K0));
      fill(F, K0, 1.0, st);
      int fb = 0;
      for (int cc = C - 1; cc >= 0; --cc) {
        const Column& K_ = S.col(cc);
        const int chl = S.A->bond[cc], chr = S.A->bond[cc + 1];
        Ft[cc] = h->ws.get<double>("srch_Ft" + std::to_string(cc), size_t(K_.nK()) * chr * K0);
        gemm(K_.Wk, false, K_.nBR(), F, false, (long long)chr * K0, Ft[cc], (long long)chr * K0, K_.nK(), chr * K0,
             K_.nBR(), 1.0, 0, st);
        if (cc > 0) {
          double* Fn = h->ws.get<double>(fb ? "srch_F1" : "srch_F0", size_t(K_.nBL()) * chl * K0);
          fb ^= 1;
          renv_step(h, r, cc, Ahat[cc], Ft[cc], fr[cc], K0, chl, chr, Fn);
          F = Fn;
        }
      }
      anc.resize(K);
      std::iota(anc.begin(), anc.end(), 0);
      E = h->ws.get<double>("srch_E" + std::to_string(ebuf), size_t(K));
      fill(E, K, 1.0, st);
    } else {
      // place column c-1: E (Kprev branches) -> E for the K survivors
      const int cc = c - 1, chl = S.A->bond[cc], chr = S.A->bond[cc + 1];
      std::vector<int32_t> xs(K);
      std::vector<int32_t> nanc(K);
      for (int k = 0; k < K; ++k) {
        xs[k] = cfg[size_t(k) * step + step - 1];
        nanc[k] = anc[par[k]];
      }
      anc.swap(nanc);
      int32_t* dpar = S.alloc<int32_t>(K);
      int32_t* dxs = S.alloc<int32_t>(K);
      SGTN_CUDA(cudaMemcpyAsync(dpar, par.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      SGTN_CUDA(cudaMemcpyAsync(dxs, xs.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      ebuf ^= 1;
      double* En = h->ws.get<double>("srch_E" + std::to_string(ebuf), size_t(S.col(cc).nBR()) * chr * K);
      lenv_step(h, r, cc, Ahat[cc], E, Kprev, K, dpar, dxs, chl, chr, En);
      E = En;
    }
    // this column's f and Ft for the current branches
    int32_t* danc = S.alloc<int32_t>(K);
    SGTN_CUDA(cudaMemcpyAsync(danc, anc.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const Column& Kc = S.col(c);
    const int chr = S.A->bond[c + 1];
    const long long frow = Kc.nU, trow = (long long)Kc.nK() * chr;
    S.f.assign(C, nullptr);
    S.f[c] = S.alloc<double>(size_t(frow) * K);
    {
      KTimer kt("gather", h->st);
      gather_cols_kernel<<<nblk(frow * K), 256, 0, st>>>(fr[c], frow, K0, danc, K, S.f[c]);
    }
    double* Ftc = S.alloc<double>(size_t(trow) * K);
    {
      KTimer kt("gather", h->st);
      gather_cols_kernel<<<nblk(trow * K), 256, 0, st>>>(Ft[c], trow, K0, danc, K, Ftc);
    }
    g_count.launches += 2;
    S.E = E;
    S.Ahat = Ahat;
    compute_scores(S, Ftc);
    ncfg.assign(size_t(M) * (step + 1), 0);
    nlp.assign(M, 0.0);
    par.assign(M, 0);
    int oc = 0;
    MergeLosers ml;
    select_step(S, step, M, cfg.data(), lp.data(), ncfg.data(), nlp.data(), &oc, &pd, par.data(),
                book ? &ml : nullptr);
    h->sync();   // the inputs of this step (host vectors) are replaced below
    if (book) book->step(step, cfg, ncfg, oc, par, ml);
    if (S.spilled) cap += 2 * S.spilled;
    cfg.assign(ncfg.begin(), ncfg.begin() + size_t(oc) * (step + 1));
    lp.assign(nlp.begin(), nlp.begin() + oc);
    par.resize(oc);
    Kprev = K;
    count = oc;
  }
  int nw = std::min(n_out, count);
  std::vector<int8_t> spins(size_t(nw) * h->M.N);
  for (int i = 0; i < nw; ++i)
    for (int s = 0; s < RC; ++s) {
      const HSite& S = h->M.sites[s];
      int64_t st = S.states[cfg[size_t(i) * RC + s]];
      for (size_t j = 0; j < S.spins.size(); ++j) spins[size_t(i) * h->M.N + S.spins[j]] = ((st >> j) & 1) ? -1 : 1;
    }
  energies(h, nw, spins.data(), out_energy);
  std::copy(spins.begin(), spins.end(), out_spins);
  for (int i = 0; i < nw; ++i) out_logp[i] = lp[i];
  *out_pd = pd;
  *out_count = nw;
  if (book && dout) {
    *dout = book->drops[0];
    std::sort(dout->begin(), dout->end(), [](const Drop& a, const Drop& b) {
      return a.dE != b.dE ? a.dE < b.dE : a.flips < b.flips;
    });
  }
}

}  // namespace sgtn
