// Double-precision kernels of the sgtn library: the segmented gathered GEMM
// that evaluates the sparse site diagrams of Fig. 7 (and plain GEMMs), the
// one-sided Jacobi SVD used for every truncation and orthonormalisation
// (Hestenes 1958; Demmel & Veselic 1992), and small helpers.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "kern.h"

namespace sgtn {

namespace {

constexpr int TK = 16;

// Segmented gathered GEMM.  One CTA (256 threads, a 16 x 16 grid) owns a
// BM x BN tile of one output segment and runs over the flattened (term,
// k-chunk) sequence of that segment: the operand tiles of the next step are
// loaded into registers while the current ones are multiplied out of shared
// memory (one barrier per step).  Thread (ty, tx) accumulates rows
// ty RM + u and columns tx RN + v of the tile (RM = BM / 16, RN = BN / 16) in
// the arithmetic type CT.  Term coefficients and column
// scales are applied to the Y tile as it is stored.  Tile loads run along
// whichever operand index has unit stride, so they coalesce.
template <class CT, int BM, int BN>
__global__ void __launch_bounds__(256) seg_gemm_kernel(SegGemm a) {
  constexpr int RM = BM / 16, RN = BN / 16;
  constexpr int XL = (BM * TK + 255) / 256, YL = (TK * BN + 255) / 256;
  // rows padded by 16 bytes: every row starts 16-byte aligned, so a thread's
  // RM (RN) contiguous tile entries come in vector loads
  constexpr int PAD = 16 / int(sizeof(CT));
  __shared__ __align__(16) CT Xs[2][TK][BM + PAD];
  __shared__ __align__(16) CT Ys[2][TK][BN + PAD];
  const int seg = blockIdx.x / a.kpart, part = blockIdx.x % a.kpart;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.z * BN;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  CT acc[RM][RN];
#pragma unroll
  for (int u = 0; u < RM; ++u)
#pragma unroll
    for (int v = 0; v < RN; ++v) acc[u][v] = CT(0);
  int t0, t1;
  long long ooff;
  int qlen = a.q;
  if (a.splitk) {
    const int k_lo = seg * a.splitk;
    qlen = min(a.splitk, a.q - k_lo);
  }
  if (a.seg_ptr) {
    t0 = a.seg_ptr[seg];
    t1 = a.seg_ptr[seg + 1];
    ooff = a.out_by_seg ? (long long)seg * a.ors : (long long)a.seg_or[seg] * a.ors + (long long)a.seg_oc[seg] * a.ocs;
  } else {
    t0 = seg;
    t1 = seg + 1;
    ooff = (long long)seg * a.ors;
  }
  if (a.kpart > 1) ooff = (long long)blockIdx.x * a.ors;   // partial block of (segment, part)
  if ((a.tri & 1) && i0 >= j0 + BN) return;   // wholly below the diagonal: not needed
  int k_base = a.splitk ? seg * a.splitk : 0;
  if (a.tri & 2) qlen = max(0, min(qlen, j0 + BN - k_base));   // Y[k][j] = 0 for k > j
  const int nk = (qlen + TK - 1) / TK;
  const int nall = (t1 - t0) * nk;
  // this CTA's share of the segment's (term, k-chunk) sequence
  const int sbeg = int((long long)nall * part / a.kpart), send = int((long long)nall * (part + 1) / a.kpart);
  const int nsteps = send - sbeg;
  const bool x_kfast = (a.xs_k == 1), y_jfast = (a.ys_j == 1);
  // per-term operand offsets and scales
  auto term = [&](int t, long long& xoff, long long& yoff, double& cf, const double*& cs) {
    cf = 1.0;
    cs = nullptr;
    if (a.seg_ptr) {
      xoff = (long long)a.xr[t] * a.xrs + (long long)a.xc[t] * a.xcs;
      yoff = (long long)a.yr[t] * a.yrs + (long long)a.yc[t] * a.ycs;
      if (a.coef) cf = a.coef[a.cidx[t]];
      if (a.cs) cs = a.cs + (long long)a.csrow[t] * a.cs_ld;
    } else if (a.splitk) {
      xoff = (long long)t * a.splitk * a.xs_k;
      yoff = (long long)t * a.splitk * a.ys_k;
    } else {
      xoff = (long long)t * a.xrs;
      yoff = (long long)t * a.yrs;
    }
  };
  CT xr[XL], yr[YL];
  auto load = [&](int lstep) {
    const int step = sbeg + lstep;
    const int t = t0 + step / nk, k0 = (step % nk) * TK;
    long long xoff, yoff;
    double cf;
    const double* cs;
    term(t, xoff, yoff, cf, cs);
#pragma unroll
    for (int l = 0; l < XL; ++l) {
      const int e = tid + l * 256;
      int ii, kk;
      if (x_kfast) ii = e / TK, kk = e % TK;
      else ii = e % BM, kk = e / BM;
      const int i = i0 + ii, k = k0 + kk;
      xr[l] = (e < BM * TK && i < a.p && k < qlen) ? CT(a.X[xoff + (long long)i * a.xs_i + (long long)k * a.xs_k]) : CT(0);
    }
#pragma unroll
    for (int l = 0; l < YL; ++l) {
      const int e = tid + l * 256;
      int kk, jj;
      if (y_jfast) kk = e / BN, jj = e % BN;
      else kk = e % TK, jj = e / TK;
      const int k = k0 + kk, j = j0 + jj;
      double v = 0.0;
      if (e < TK * BN && k < qlen && j < a.s) {
        v = cf * a.Y[yoff + (long long)k * a.ys_k + (long long)j * a.ys_j];
        if (cs) v *= cs[j];
      }
      yr[l] = CT(v);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int l = 0; l < XL; ++l) {
      const int e = tid + l * 256;
      if (e >= BM * TK) break;
      int ii, kk;
      if (x_kfast) ii = e / TK, kk = e % TK;
      else ii = e % BM, kk = e / BM;
      Xs[buf][kk][ii] = xr[l];
    }
#pragma unroll
    for (int l = 0; l < YL; ++l) {
      const int e = tid + l * 256;
      if (e >= TK * BN) break;
      int kk, jj;
      if (y_jfast) kk = e / BN, jj = e % BN;
      else kk = e % TK, jj = e / TK;
      Ys[buf][kk][jj] = yr[l];
    }
  };
  if (nsteps > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int step = 0; step < nsteps; ++step) {
    const int buf = step & 1;
    if (step + 1 < nsteps) load(step + 1);   // global loads in flight during the FMAs
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      CT xv[RM], yv[RN];
#pragma unroll
      for (int u = 0; u < RM; ++u) xv[u] = Xs[buf][kk][ty * RM + u];
#pragma unroll
      for (int v = 0; v < RN; ++v) yv[v] = Ys[buf][kk][tx * RN + v];
#pragma unroll
      for (int u = 0; u < RM; ++u)
#pragma unroll
        for (int v = 0; v < RN; ++v) acc[u][v] = fma(xv[u], yv[v], acc[u][v]);
    }
    if (step + 1 < nsteps) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < RM; ++u) {
    const int i = i0 + ty * RM + u;
    if (i >= a.p) continue;
#pragma unroll
    for (int v = 0; v < RN; ++v) {
      const int j = j0 + tx * RN + v;
      if (j >= a.s) continue;
      double* o = a.O + ooff + (long long)i * a.os_i + (long long)j * a.os_j;
      const double val = a.alpha * double(acc[u][v]);
      *o = a.accumulate ? *o + val : val;
    }
  }
}

// Sum of the kpart partial blocks P[seg * kpart + part] (p x s, row-major) of
// each segment, in part order, into the segment's output block.
__global__ void kpart_reduce_kernel(const double* P, int nseg, int kpart, int p, int s, SegGemm a) {
  const long long blk = (long long)p * s, total = (long long)nseg * blk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = int(e / blk);
    const long long r = e % blk;
    const int i = int(r / s), j = int(r % s);
    double v = 0.0;
    for (int q = 0; q < kpart; ++q) v += P[((long long)g * kpart + q) * blk + r];
    long long ooff;
    if (a.seg_ptr)
      ooff = a.out_by_seg ? (long long)g * a.ors : (long long)a.seg_or[g] * a.ors + (long long)a.seg_oc[g] * a.ocs;
    else
      ooff = (long long)g * a.ors;
    double* o = a.O + ooff + (long long)i * a.os_i + (long long)j * a.os_j;
    *o = a.accumulate ? *o + a.alpha * v : a.alpha * v;
  }
}

// Sum of the virtual-segment blocks P[v] (p x s, row-major) of each segment,
// in virtual-segment order, into the segment's output block.
__global__ void seg_reduce_kernel(const double* P, const int32_t* vfirst, int nseg, int p, int s, SegGemm a) {
  const long long blk = (long long)p * s, total = (long long)nseg * blk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = int(e / blk);
    const long long r = e % blk;
    const int i = int(r / s), j = int(r % s);
    double v = 0.0;
    for (int q = vfirst[g]; q < vfirst[g + 1]; ++q) v += P[q * blk + r];
    const long long ooff =
        a.out_by_seg ? (long long)g * a.ors : (long long)a.seg_or[g] * a.ors + (long long)a.seg_oc[g] * a.ocs;
    double* o = a.O + ooff + (long long)i * a.os_i + (long long)j * a.os_j;
    *o = a.accumulate ? *o + a.alpha * v : a.alpha * v;
  }
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Single-CTA cyclic one-sided Jacobi with a round-robin pairing.  Columns
// whose squared norm is below (eps * ||X||_F)^2 are numerically zero: they are
// never rotated (they would otherwise trade rounding noise forever) and the
// caller drops them with the rank rule.
__device__ void jacobi_body(double* X, int len, int p, long long si, long long sj, double* V, int max_sweeps,
                            double tol, int* status) {
  __shared__ int rotated;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (V)
    for (long long e = threadIdx.x; e < (long long)p * p; e += blockDim.x)
      V[e] = ((e / p) == (e % p)) ? 1.0 : 0.0;
  // ||X||_F^2
  double fro = 0;
  for (long long e = threadIdx.x; e < (long long)len * p; e += blockDim.x) {
    double v = X[(e % len) * si + (e / len) * sj];
    fro = fma(v, v, fro);
  }
  fro = warp_sum(fro);
  if (lane == 0) red[warp] = fro;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  const double zero2 = red[0] * 1e-30;   // (1e-15 ||X||_F)^2
  const int pp = p + (p & 1);
  int sweep = 0;
  bool done = (p < 2);
  __syncthreads();
  while (!done && sweep < max_sweeps) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int t = 0; t < pp - 1; ++t) {
      for (int w = warp; w < pp / 2; w += nwarp) {
        int pa = w, pb = pp - 1 - w;
        int ca = pa == 0 ? 0 : 1 + (pa - 1 + t) % (pp - 1);
        int cb = pb == 0 ? 0 : 1 + (pb - 1 + t) % (pp - 1);
        if (ca >= p || cb >= p) continue;
        double* xa = X + ca * sj;
        double* xb = X + cb * sj;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < len; i += 32) {
          double u = xa[i * si], v = xb[i * si];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > zero2 && be > zero2 && fabs(ga) > tol * sqrt(al * be)) {
          double zeta = (be - al) / (2.0 * ga);
          double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
          for (int i = lane; i < len; i += 32) {
            double u = xa[i * si], v = xb[i * si];
            xa[i * si] = c * u - s * v;
            xb[i * si] = s * u + c * v;
          }
          if (V) {
            double* va = V + (long long)ca * p;
            double* vb = V + (long long)cb * p;
            for (int i = lane; i < p; i += 32) {
              double u = va[i], v = vb[i];
              va[i] = c * u - s * v;
              vb[i] = s * u + c * v;
            }
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    ++sweep;
    done = (rotated == 0);
    __syncthreads();
  }
  if (threadIdx.x == 0) status[0] = done ? sweep : -1;
}


// Same, with the matrix (and V) staged in shared memory, column-major.
__global__ void __launch_bounds__(1024) jacobi_smem_kernel(double* X, int len, int p, long long si, long long sj,
                                                           double* V, int max_sweeps, double tol, int* status) {
  extern __shared__ double sm[];
  double* Xs = sm;
  double* Vs = V ? sm + (long long)len * p : nullptr;
  for (long long e = threadIdx.x; e < (long long)len * p; e += blockDim.x) {
    long long j = e / len, i = e % len;
    Xs[e] = X[i * si + j * sj];
  }
  __syncthreads();
  jacobi_body(Xs, len, p, 1, len, Vs, max_sweeps, tol, status);
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)len * p; e += blockDim.x) {
    long long j = e / len, i = e % len;
    X[i * si + j * sj] = Xs[e];
  }
  if (V)
    for (long long e = threadIdx.x; e < (long long)p * p; e += blockDim.x) V[e] = Vs[e];
}

// Thread-block-cluster variant: the p vectors are spread over the shared
// memories of the cluster's P CTAs (vector j in CTA j % P, slot j / P, with
// its column of V beside it).  In each round-robin step the warps of all CTAs
// rotate disjoint pairs, reading and writing both vectors through distributed
// shared memory, and a cluster barrier closes the step.  Pairs, rotations and
// the stopping rule are those of jacobi_body; the FP64 work of a step is spread
// over P SMs instead of one.
// RV > 0: vectors of at most 32 RV elements stay in registers between the dot
// products and the rotation (one distributed-shared-memory round trip a pair).
template <int RV>
__global__ void __launch_bounds__(512) jacobi_cluster_kernel(double* X, int len, int p, long long si, long long sj,
                                                              double* V, int max_sweeps, double tol, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double csm[];
  __shared__ double red[32];
  __shared__ double fro_part;
  __shared__ int flag[2];
  const int P = int(cl.num_blocks()), rank = int(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int slots = (p + P - 1) / P;
  double* Xs = csm;                                   // slots x len
  double* Vs = V ? csm + (long long)slots * len : nullptr;   // slots x p
  double* Ns = csm + (long long)slots * len + (V ? (long long)slots * p : 0);   // slots: squared norms
  double f = 0;
  for (int l = 0; l < slots; ++l) {
    const int j = l * P + rank;
    if (j >= p) break;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      double v = X[i * si + j * sj];
      Xs[(long long)l * len + i] = v;
      f = fma(v, v, f);
    }
    if (Vs)
      for (int i = threadIdx.x; i < p; i += blockDim.x) Vs[(long long)l * p + i] = (i == j) ? 1.0 : 0.0;
  }
  f = warp_sum(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    fro_part = t;
  }
  cl.sync();
  double fro = 0;
  for (int r = 0; r < P; ++r) fro += *cl.map_shared_rank(&fro_part, r);
  const double zero2 = fro * 1e-30;   // (1e-15 ||X||_F)^2
  const int pp = p + (p & 1), npair = pp / 2;
  int sweep = 0;
  bool done = (p < 2);
  const double tol2 = tol * tol;
  while (!done && sweep < max_sweeps) {
    int rot = 0;
    // exact squared norms at the start of every sweep; within the sweep they
    // follow the rotations (a' = a - t g, b' = b + t g, t = tan of the angle)
    for (int l = warp; l < slots; l += nwarp) {
      if (l * P + rank >= p) continue;
      double q = 0;
      for (int i = lane; i < len; i += 32) q = fma(Xs[(long long)l * len + i], Xs[(long long)l * len + i], q);
      q = warp_sum(q);
      if (lane == 0) Ns[l] = q;
    }
    cl.sync();
    for (int t = 0; t < pp - 1; ++t) {
      for (int w = rank + P * warp; w < npair; w += P * nwarp) {
        int pa = w, pb = pp - 1 - w;
        int ca = pa == 0 ? 0 : 1 + (pa - 1 + t) % (pp - 1);
        int cb = pb == 0 ? 0 : 1 + (pb - 1 + t) % (pp - 1);
        if (ca >= p || cb >= p) continue;
        double* xa = cl.map_shared_rank(Xs + (long long)(ca / P) * len, ca % P);
        double* xb = cl.map_shared_rank(Xs + (long long)(cb / P) * len, cb % P);
        double* na = cl.map_shared_rank(Ns + ca / P, ca % P);
        double* nb = cl.map_shared_rank(Ns + cb / P, cb % P);
        const double al = *na, be = *nb;
        double ga = 0;
        double ur[RV > 0 ? RV : 1], vr[RV > 0 ? RV : 1];
        if constexpr (RV > 0) {
#pragma unroll
          for (int q = 0; q < RV; ++q) {
            const int i = lane + 32 * q;
            ur[q] = i < len ? xa[i] : 0.0;
            vr[q] = i < len ? xb[i] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < RV; ++q) ga = fma(ur[q], vr[q], ga);
        } else {
          for (int i = lane; i < len; i += 32) ga = fma(xa[i], xb[i], ga);
        }
        ga = warp_sum(ga);
        if (al > zero2 && be > zero2 && ga * ga > tol2 * al * be) {
          // angle that zeroes the pair's product: with d = b - a and
          // r = sqrt(d^2 + 4 g^2), cos^2 = (1 + |d| / r) / 2 and
          // sin = sign(d) g / (r cos); tan = sin / cos
          const double d = be - al;
          const double rinv = rsqrt(fma(d, d, 4.0 * ga * ga));
          const double c2 = fma(0.5 * fabs(d), rinv, 0.5);
          const double rc = rsqrt(c2);
          const double c = c2 * rc, s = (d >= 0 ? 1.0 : -1.0) * ga * rinv * rc;
          const double tg = s * rc;
          double an = al - tg * ga, bn = be + tg * ga;
          if constexpr (RV > 0) {
#pragma unroll
            for (int q = 0; q < RV; ++q) {
              const int i = lane + 32 * q;
              const double u = ur[q], v = vr[q];
              ur[q] = c * u - s * v;
              vr[q] = s * u + c * v;
              if (i < len) {
                xa[i] = ur[q];
                xb[i] = vr[q];
              }
            }
            if (an < 1e-4 * al || bn < 1e-4 * be) {
              // cancellation in the update: recompute both norms
              double qa = 0, qb = 0;
#pragma unroll
              for (int q = 0; q < RV; ++q) {
                qa = fma(ur[q], ur[q], qa);
                qb = fma(vr[q], vr[q], qb);
              }
              an = warp_sum(qa);
              bn = warp_sum(qb);
            }
          } else {
            double qa = 0, qb = 0;
            for (int i = lane; i < len; i += 32) {
              const double u = xa[i], v = xb[i];
              const double u2 = c * u - s * v, v2 = s * u + c * v;
              xa[i] = u2;
              xb[i] = v2;
              qa = fma(u2, u2, qa);
              qb = fma(v2, v2, qb);
            }
            if (an < 1e-4 * al || bn < 1e-4 * be) {
              an = warp_sum(qa);
              bn = warp_sum(qb);
            }
          }
          if (lane == 0) {
            *na = an;
            *nb = bn;
          }
          if (Vs) {
            double* va = cl.map_shared_rank(Vs + (long long)(ca / P) * p, ca % P);
            double* vb = cl.map_shared_rank(Vs + (long long)(cb / P) * p, cb % P);
            for (int i = lane; i < p; i += 32) {
              double u = va[i], v = vb[i];
              va[i] = c * u - s * v;
              vb[i] = s * u + c * v;
            }
          }
          rot = 1;
        }
      }
      cl.sync();
    }
    int any_local = __syncthreads_or(rot);
    if (threadIdx.x == 0) flag[sweep & 1] = any_local;
    cl.sync();
    int any = 0;
    for (int r = 0; r < P; ++r) any |= *cl.map_shared_rank(&flag[sweep & 1], r);
    ++sweep;
    done = (any == 0);
  }
  for (int l = 0; l < slots; ++l) {
    const int j = l * P + rank;
    if (j >= p) break;
    for (int i = threadIdx.x; i < len; i += blockDim.x) X[i * si + j * sj] = Xs[(long long)l * len + i];
    if (V)
      for (int i = threadIdx.x; i < p; i += blockDim.x) V[(long long)j * p + i] = Vs[(long long)l * p + i];
  }
  if (rank == 0 && threadIdx.x == 0) status[0] = done ? sweep : -1;
  cl.sync();   // no CTA leaves while another may still read its flags
}

// Cooperative multi-CTA variant for many columns: one warp rotates one pair
// per round, rounds are separated by grid-wide barriers (the launch is
// cooperative, so all CTAs are resident).  flags[s] counts rotations in sweep
// s and must be zero on entry.
__global__ void __launch_bounds__(128) jacobi_coop_kernel(double* X, int len, int p, long long si, long long sj,
                                                          double* V, int max_sweeps, double tol, int* status,
                                                          int* flags, double* fro_out) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + warp, ngw = gridDim.x * nw;
  if (V)
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)p * p;
         e += (long long)gridDim.x * blockDim.x)
      V[e] = ((e / p) == (e % p)) ? 1.0 : 0.0;
  if (blockIdx.x == 0) {
    double f = 0;
    for (long long e = threadIdx.x; e < (long long)len * p; e += blockDim.x) {
      double v = X[(e % len) * si + (e / len) * sj];
      f = fma(v, v, f);
    }
    f = warp_sum(f);
    if (lane == 0) red[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < nw; ++w) t += red[w];
      fro_out[0] = t;
    }
  }
  grid.sync();
  const double zero2 = fro_out[0] * 1e-30;
  const int pp = p + (p & 1);
  int sweep = 0;
  bool done = (p < 2);
  while (!done && sweep < max_sweeps) {
    for (int t = 0; t < pp - 1; ++t) {
      for (int w = gw; w < pp / 2; w += ngw) {
        int pa = w, pb = pp - 1 - w;
        int ca = pa == 0 ? 0 : 1 + (pa - 1 + t) % (pp - 1);
        int cb = pb == 0 ? 0 : 1 + (pb - 1 + t) % (pp - 1);
        if (ca >= p || cb >= p) continue;
        double* xa = X + ca * sj;
        double* xb = X + cb * sj;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < len; i += 32) {
          double u = xa[i * si], v = xb[i * si];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > zero2 && be > zero2 && fabs(ga) > tol * sqrt(al * be)) {
          double zeta = (be - al) / (2.0 * ga);
          double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
          for (int i = lane; i < len; i += 32) {
            double u = xa[i * si], v = xb[i * si];
            xa[i * si] = c * u - s * v;
            xb[i * si] = s * u + c * v;
          }
          if (V) {
            double* va = V + (long long)ca * p;
            double* vb = V + (long long)cb * p;
            for (int i = lane; i < p; i += 32) {
              double u = va[i], v = vb[i];
              va[i] = c * u - s * v;
              vb[i] = s * u + c * v;
            }
          }
          if (lane == 0) atomicAdd(flags + sweep, 1);
        }
      }
      grid.sync();
    }
    done = (atomicAdd(flags + sweep, 0) == 0);
    ++sweep;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) status[0] = done ? sweep : -1;
}

// Right-looking upper Cholesky of the n x n block W + shift I in shared memory
// (two barriers a column: the scaled pivot row is staged, then the trailing
// upper triangle is updated by a 32 x 32 thread grid), then R^{-1}
// right-looking from the last row (R X = I: finished row j of X is subtracted
// from every row above it), with X kept transposed in the free lower
// triangle.  W, R and Rinv are blocks of row-major matrices with leading
// dimension ld; Rinv may alias W (all of W is read before anything is
// written).  Gd points at the matching diagonal block of the original G (for
// the pivot ratios).  On a non-positive pivot j the first failure is recorded
// as status[0] = status_off + j + 1; status is not written otherwise.
// minratio[0] = min(minratio[0], smallest pivot / (G_jj + shift)).  T is the
// arithmetic type (float: a cheap factor whose rounding a later FP64 pass
// removes); memory stays FP64.
__device__ __forceinline__ float chol_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double chol_rsqrt(double x) { return rsqrt(x); }

template <class T>
__global__ void __launch_bounds__(1024) cholesky_inv_kernel(const double* W, int n, int ld, double shift, double* R,
                                                            double* Rinv, const double* Gd, int* status,
                                                            int status_off, double* minratio, int init) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T* A = reinterpret_cast<T*>(chol_smem);   // n x n
  T* row = A + n * n;                       // n: staged row / 1 / R_jj
  T* gd = row + n;                          // n: 1 / diagonal of G + shift I
  __shared__ int fail;
  __shared__ T piv[2];   // sqrt of the current pivot and its reciprocal
  __shared__ double mr;  // smallest pivot / (diagonal of G + shift)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    A[e] = j >= i ? T(W[(long long)i * ld + j] + (i == j ? shift : 0.0)) : T(0);
  }
  // reciprocals of the diagonal of G + shift I, all in parallel: a division
  // (about 640 cycles of dependent FP64 latency on B300) stays off the chain
  // of pivots, which is the kernel's critical path
  for (int i = threadIdx.x; i < n; i += blockDim.x) gd[i] = T(1.0 / (Gd[(long long)i * (ld + 1)] + shift));
  __syncthreads();
  // thread 0 takes each pivot: one reciprocal square root (the pivot's square
  // root is d times it) instead of a square root followed by a division
  auto take_pivot = [&](int j) {
    const T d = A[j * n + j];
    const bool bad = !(d > T(0));
    if (bad && !fail) fail = j + 1;
    mr = fmin(mr, double(d * gd[j]));
    const T ri = bad ? T(1) : chol_rsqrt(d);
    piv[1] = ri;
    piv[0] = bad ? T(1) : d * ri;
  };
  if (threadIdx.x == 0) {
    fail = 0;
    mr = 1.0;
    if (n > 0) take_pivot(0);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const T r = piv[0], ri = piv[1];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) row[i] = A[j * n + i] * ri;
    __syncthreads();
    if (threadIdx.x == 0) A[j * n + j] = r;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[j * n + i] = row[i];
    for (int k = j + 1 + ty; k < n; k += 32) {
      const T rk = row[k];
      for (int i = k + tx; i < n; i += 32) A[k * n + i] -= rk * row[i];
    }
    // element (j+1, j+1) was updated by thread 0 (k = j+1, i = k): next pivot
    if (threadIdx.x == 0 && j + 1 < n) take_pivot(j + 1);
    __syncthreads();
  }
  // R^{-1} = X (upper): X[i][c] (i < c) lives at A[c * n + i]; X[i][i] = 1 / R_ii
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = T(1) / A[i * n + i];
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    // row j of X is final once scaled by 1 / R_jj
    for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) A[c * n + j] *= row[j];
    __syncthreads();
    // rows k < j:  X[k][c] -= R[k][j] X[j][c]  for c >= j
    for (int k = ty; k < j; k += 32) {
      const T rkj = A[k * n + j];
      for (int c = j + tx; c < n; c += 32) {
        const T xjc = (c == j) ? row[j] : A[c * n + j];
        A[c * n + k] -= rkj * xjc;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e % n;
    R[(long long)i * ld + c] = c >= i ? double(A[e]) : 0.0;
    Rinv[(long long)i * ld + c] = c > i ? double(A[c * n + i]) : (c == i ? double(row[i]) : 0.0);
  }
  if (threadIdx.x == 0) {
    // the first diagonal block of a factorisation starts both outputs afresh
    if (init) status[0] = fail ? status_off + fail : 0;
    else if (fail && status[0] == 0) status[0] = status_off + fail;
    if (minratio) minratio[0] = init ? mr : fmin(minratio[0], mr);
  }
}

// Statistics of the upper triangle of a k x k Gram matrix, one CTA:
// out[0] = max |G_ij - delta_ij| over j >= i (NaN if an entry is not finite),
// out[1] = trace.  Fixed-order reductions.
__global__ void __launch_bounds__(1024) gram_stats_kernel(const double* G, int k, double* out) {
  __shared__ double rmax[32], rsum[32];
  __shared__ int rbad[32];
  double mx = 0.0, tr = 0.0;
  int bad = 0;
  for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
    const int i = int(e / k), j = int(e % k);
    if (j < i) continue;
    const double g = G[e];
    if (!isfinite(g)) bad = 1;
    mx = fmax(mx, fabs(g - (i == j ? 1.0 : 0.0)));
    if (i == j) tr += g;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    rmax[warp] = mx;
    rsum[warp] = tr;
    rbad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, t = 0.0;
    int b = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      m = fmax(m, rmax[w]);
      t += rsum[w];
      b |= rbad[w];
    }
    out[0] = b ? nan("") : m;
    out[1] = t;
  }
}

// X[i][j] = 0 and Y[i][j] = 0 for two rows x cols blocks with leading dimension ld
__global__ void zero_blocks2_kernel(double* X, double* Y, int rows, int cols, int ld) {
  const long long n = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long o = (e / cols) * ld + e % cols;
    X[o] = 0.0;
    Y[o] = 0.0;
  }
}


// Cholesky with diagonal pivoting of a positive semidefinite G (n x n, FP64),
// stopped at the numerical rank: step j takes the largest remaining diagonal
// of the Schur complement and stops when it is <= max(tol_rel * max diag(G),
// tol_abs).  Out: rank r, perm[0..r) (the pivot order), R (r x r upper, row-major
// with leading dimension n) with G[perm][perm] ~ R^T R on the leading r x r
// block, and R^{-1} (same layout).
__global__ void __launch_bounds__(1024) pchol_inv_kernel(const double* G, int n, double tol_rel, double tol_abs,
                                                         double* R, double* Rinv, int32_t* perm, int* rank) {
  extern __shared__ double A[];   // n x n, original indexing
  __shared__ int piv[256];
  __shared__ double dmax0;
  __shared__ int rk, qsel;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = G[e];
  for (int i = threadIdx.x; i < n; i += blockDim.x) piv[i] = i;
  __syncthreads();
  if (warp == 0) {
    double m = 0;
    for (int i = lane; i < n; i += 32) m = fmax(m, A[i * n + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      dmax0 = m;
      rk = n;
    }
  }
  __syncthreads();
  const double stop = fmax(tol_rel * dmax0, tol_abs);
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      // argmax of the remaining diagonal (ties: lowest position)
      double bv = -1.0;
      int bi = n;
      for (int i = j + lane; i < n; i += 32) {
        double v = A[piv[i] * n + piv[i]];
        if (v > bv) bv = v, bi = i;
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) bv = ov, bi = oi;
      }
      if (lane == 0) {
        if (!(bv > stop)) {
          rk = j;
          qsel = -1;
        } else {
          int t = piv[j];
          piv[j] = piv[bi];
          piv[bi] = t;
          A[piv[j] * n + piv[j]] = sqrt(bv);
          qsel = bi;
        }
      }
    }
    __syncthreads();
    if (qsel < 0) break;
    const int pj = piv[j];
    const double r = A[pj * n + pj];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[pj * n + piv[i]] /= r;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int a = piv[j + 1 + e / m], b = piv[j + 1 + e % m];
      A[a * n + b] -= A[pj * n + a] * A[pj * n + b];
    }
    __syncthreads();
  }
  const int r = rk;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, k = e % r;
    R[i * n + k] = k >= i ? A[piv[i] * n + piv[k]] : 0.0;
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) perm[i] = piv[i];
  __syncthreads();
  // R X = I by back substitution, one column per thread (R read from global)
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = r - 1; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) v -= A[piv[i] * n + piv[k]] * Rinv[k * n + c];
      Rinv[i * n + c] = (i <= c) ? v / A[piv[i] * n + piv[i]] : 0.0;
    }
  }
  if (threadIdx.x == 0) rank[0] = r;
}

__global__ void vec_norms_kernel(const double* X, int len, int p, long long si, long long sj, double* out) {
  int j = blockIdx.x;
  double a = 0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    double v = X[i * si + j * sj];
    a = fma(v, v, a);
  }
  __shared__ double red[32];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    b = warp_sum(b);
    if (threadIdx.x == 0) out[j] = sqrt(b);
  }
}

__global__ void gather_vecs_kernel(const double* X, int len, long long si, long long sj, const int32_t* perm,
                                   const double* scale, int k, double* out, long long oi, long long oj) {
  long long n = (long long)len * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int jj = int(e / len), i = int(e % len);
    out[i * oi + jj * oj] = scale[jj] * X[i * si + (long long)perm[jj] * sj];
  }
}

__global__ void permute3_kernel(const double* in, int A, int B, int Cd, double* out) {
  long long n = (long long)A * B * Cd;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int c = int(e % Cd);
    long long r = e / Cd;
    int b = int(r % B), a = int(r / B);
    out[((long long)b * A + a) * Cd + c] = in[e];
  }
}

struct PermArgs {
  int nd;
  long long in_stride[6];    // stride in `in` of each OUTPUT axis
  long long out_dim[6];
};

__global__ void permute_nd_kernel(const double* in, double* out, long long n, PermArgs pa) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    long long rem = e, src = 0;
    for (int k = pa.nd - 1; k >= 0; --k) {
      long long ik = rem % pa.out_dim[k];
      rem /= pa.out_dim[k];
      src += ik * pa.in_stride[k];
    }
    out[e] = in[src];
  }
}

__global__ void scatter_blocks_kernel(const double* blocks, long long total, int chl, int kp, const int32_t* seg_bl,
                                      const int32_t* seg_u, double* dense, long long n) {
  const long long blk = (long long)chl * kp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long sgi = e / blk, r = e % blk;
    long long i = r / kp, j = r % kp;
    dense[((long long)seg_bl[sgi] * chl + i) * n + (long long)seg_u[sgi] * kp + j] = blocks[e];
  }
}

__global__ void fro_norm_kernel(const double* x, long long n, double* out) {
  __shared__ double red[32];
  double a = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) a = fma(x[i], x[i], a);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    b = warp_sum(b);
    if (threadIdx.x == 0) out[0] = sqrt(b);
  }
}

__global__ void scale_by_inv_kernel(double* x, long long n, const double* norm) {
  double s = 1.0 / norm[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= s;
}

// O = alpha * sum_t P[t] (+ O)
__global__ void splitk_reduce_kernel(const double* P, int nsplit, long long mn, int n, double* O, long long ldo,
                                     double alpha, int accumulate) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn; e += (long long)gridDim.x * blockDim.x) {
    double v = 0;
    for (int t = 0; t < nsplit; ++t) v += P[t * mn + e];
    double* o = O + (e / n) * ldo + (e % n);
    *o = accumulate ? *o + alpha * v : alpha * v;
  }
}

__global__ void pseudo_random_kernel(double* x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

__global__ void add_cols_kernel(double* R, const double* Q, int rows, int k, int ldq) {
  long long n = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / k, j = e % k;
    R[e] += Q[i * ldq + j];
  }
}

__global__ void scale_pow2_kernel(double* x, long long n, int e) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = ldexp(x[i], -e);
}

__global__ void fill_kernel(double* x, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void copy_kernel(double* d, const double* s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = s[i];
}

__global__ void boltzmann_kernel(const int64_t* E, long long n, int64_t Emin, double bd, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = exp(-bd * double(E[i] - Emin));
}

__global__ void build_Wa_kernel(double* Wa, int nPd, int nE, int nG, int nSig, const int32_t* s_pu,
                                const int32_t* s_pul, const int32_t* s_pur, const double* Bv, int bv_nb,
                                const double* Bdl, int bdl_nb) {
  long long n = (long long)nPd * nE * nG * nSig;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int sg = int(e % nSig);
    long long r = e / nSig;
    int g = int(r % nG);
    r /= nG;
    int ee = int(r % nE);
    int pd = int(r / nE);
    double v = 0.0;
    if (s_pul[sg] == g) v = Bv[(long long)pd * bv_nb + s_pu[sg]] * Bdl[(long long)ee * bdl_nb + s_pur[sg]];
    Wa[e] = v;
  }
}

__global__ void build_Wk_kernel(double* Wk, int nPr, int nE, int nPdr, int nLR, int nGR, const int32_t* l_pl,
                                const int32_t* l_pdl, const double* Bh, int bh_nb, const double* Bdr, int bdr_nb) {
  long long nBR = (long long)nLR * nGR;
  long long n = (long long)nPr * nE * nPdr * nBR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    long long br = e % nBR;
    long long r = e / nBR;
    int pdr = int(r % nPdr);
    r /= nPdr;
    int ee = int(r % nE);
    int pr = int(r / nE);
    int lam = int(br / nGR), gp = int(br % nGR);
    double v = 0.0;
    if (l_pdl[lam] == ee) v = Bh[(long long)pr * bh_nb + l_pl[lam]] * Bdr[(long long)pdr * bdr_nb + gp];
    Wk[e] = v;
  }
}

inline int blocks_for(long long n, int t = 256) {
  long long b = (n + t - 1) / t;
  if (b < 1) b = 1;
  if (b > 148 * 32) b = 148 * 32;
  return int(b);
}

}  // namespace

Counters g_count;

namespace {
std::mutex g_scratch_mu;
std::map<std::pair<cudaStream_t, int>, std::pair<void*, size_t>> g_scratch;
}  // namespace

void* stream_scratch(cudaStream_t st, int slot, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto& e = g_scratch[{st, slot}];
  if (bytes <= e.second) return e.first;
  if (g_no_alloc) return nullptr;
  if (e.first) {
    cudaStreamSynchronize(st);
    cudaFree(e.first);
    e = {nullptr, 0};
  }
  if (lib_malloc(&e.first, bytes) != cudaSuccess) {
    e = {nullptr, 0};
    throw SgtnError(-3, "out of device memory for " + std::to_string(bytes) + " bytes of scratch");
  }
  e.second = bytes;
  return e.first;
}

void stream_scratch_release(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  for (auto it = g_scratch.begin(); it != g_scratch.end();) {
    if (it->first.first == st) {
      cudaStreamSynchronize(st);
      cudaFree(it->second.first);
      it = g_scratch.erase(it);
    } else {
      ++it;
    }
  }
}

namespace {
struct Pending {
  std::string name;
  cudaEvent_t a, b;
  double flops;
};
struct TimerState {
  std::atomic<bool> on{false};
  std::mutex mu;                                       // guards the members below
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::array<double, 3>> acc;   // ms, launches, flops
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void resolve() {
    for (auto& p : pending) {
      cudaEventSynchronize(p.b);
      float ms = 0;
      cudaEventElapsedTime(&ms, p.a, p.b);
      auto& v = acc[p.name];
      v[0] += ms;
      v[1] += 1;
      v[2] += p.flops;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};
TimerState g_timer;
// Timers nest per host thread: only the outermost one records (a Cholesky's
// time includes its GEMMs, which are then not booked a second time).
thread_local int t_timer_depth = 0;
thread_local const char* t_timer_cur = nullptr;
thread_local cudaEvent_t t_timer_a = nullptr;
}  // namespace

void ktimer_begin(const char* name, cudaStream_t st) {
  if (!g_timer.on) return;
  if (t_timer_depth++ > 0) return;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  t_timer_cur = name;
  t_timer_a = g_timer.get();
  cudaEventRecord(t_timer_a, st);
}
void ktimer_end(cudaStream_t st, double flops) {
  if (!g_timer.on) return;
  if (t_timer_depth > 0 && --t_timer_depth > 0) return;
  if (!t_timer_cur) return;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  cudaEvent_t b = g_timer.get();
  cudaEventRecord(b, st);
  g_timer.pending.push_back({t_timer_cur, t_timer_a, b, flops});
  t_timer_cur = nullptr;
  if (g_timer.pending.size() > 4096) g_timer.resolve();
}
void ktimer_add_flops(const char* name, double flops) {
  if (!g_timer.on) return;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.acc[name][2] += flops;
}
void ktimer_enable(bool on) {
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.resolve();
  g_timer.on = on;
  t_timer_depth = 0;
  t_timer_cur = nullptr;
}
void ktimer_reset() {
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.resolve();
  g_timer.acc.clear();
}
bool ktimer_read(const char* name, double* ms, long long* n, double* flops) {
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.resolve();
  auto it = g_timer.acc.find(name);
  if (it == g_timer.acc.end()) return false;
  *ms = it->second[0];
  *n = (long long)it->second[1];
  *flops = it->second[2];
  return true;
}
std::string ktimer_names() {
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.resolve();
  std::string o;
  for (auto& kv : g_timer.acc) o += kv.first + ",";
  return o;
}

namespace {
void launch_seg(const SegGemm& a_in, cudaStream_t st, bool tc) {
  if (tc && seg_mma(a_in, st)) return;
  SegGemm a = a_in;
  // tile shape from the block shape: rows 16 / 32 / 64, columns 32 / 64
  const int bm = a.tile_m ? a.tile_m : a.p <= 16 ? 16 : a.p <= 32 ? 32 : 64;
  const int bn = a.tile_n ? a.tile_n : a.s <= 32 ? 32 : 64;
  const long long tiles = (long long)((a.p + bm - 1) / bm) * ((a.s + bn - 1) / bn);
  // A grid of fewer CTAs than two per SM leaves most of the GPU idle (B300's
  // FP64 rate per SM is low, so one long segment on one SM takes long): cut
  // each segment's (term, k-chunk) sequence into parts of at least four steps,
  // one CTA each, into scratch blocks summed afterwards in part order.
  int kpart = 1;
  double* part = nullptr;
  if (!a.splitk && !a.tri && !g_no_alloc) {
    const long long ctas = (long long)a.nseg * tiles;
    const double steps = (a.seg_ptr ? double(a.nterm) / a.nseg : 1.0) * ((a.q + TK - 1) / TK);
    if (ctas < 296 && steps >= 8) {
      kpart = int(std::min<double>({double((296 + ctas - 1) / ctas), steps / 4.0, 64.0}));
      if (kpart >= 2)
        part = static_cast<double*>(
            stream_scratch(st, SC_KPART, size_t(kpart) * a.nseg * a.p * a.s * sizeof(double)));
      if (!part) kpart = 1;
    }
  }
  SegGemm b = a;
  if (kpart > 1) {
    b.kpart = kpart;
    b.O = part;
    b.os_i = a.s;
    b.os_j = 1;
    b.ors = (long long)a.p * a.s;
    b.alpha = 1.0;
    b.accumulate = 0;
  }
  dim3 grid(a.nseg * kpart, (a.p + bm - 1) / bm, (a.s + bn - 1) / bn);
  auto go = [&](auto kern) { kern<<<grid, 256, 0, st>>>(b); };
  if (a.f32) {
    if (bm == 16) bn == 32 ? go(seg_gemm_kernel<float, 16, 32>) : go(seg_gemm_kernel<float, 16, 64>);
    else if (bm == 32) bn == 32 ? go(seg_gemm_kernel<float, 32, 32>) : go(seg_gemm_kernel<float, 32, 64>);
    else bn == 32 ? go(seg_gemm_kernel<float, 64, 32>) : go(seg_gemm_kernel<float, 64, 64>);
  } else {
    if (bm == 16) bn == 32 ? go(seg_gemm_kernel<double, 16, 32>) : go(seg_gemm_kernel<double, 16, 64>);
    else if (bm == 32) bn == 32 ? go(seg_gemm_kernel<double, 32, 32>) : go(seg_gemm_kernel<double, 32, 64>);
    else bn == 32 ? go(seg_gemm_kernel<double, 64, 32>) : go(seg_gemm_kernel<double, 64, 64>);
  }
  ++g_count.launches;
  if (kpart > 1) {
    const long long total = (long long)a.nseg * a.p * a.s;
    const int nb = int(std::min<long long>((total + 255) / 256, 148 * 16));
    kpart_reduce_kernel<<<nb, 256, 0, st>>>(part, a.nseg, kpart, a.p, a.s, a);
    ++g_count.launches;
  }
}
}  // namespace

void seg_gemm(const SegGemm& a_in, cudaStream_t st) {
  SegGemm a = a_in;
  if (g_compute_f32) a.f32 = 1;
  if (a.nseg <= 0 || a.p <= 0 || a.s <= 0) return;
  double fl = 2.0 * a.p * a.q * a.s * double(a.seg_ptr ? a.nterm : (a.splitk ? 1 : a.nseg));
  // TF32 mode: row-major gathered blocks go to the tensor cores (3xTF32)
  const bool tc = a.f32 && g_use_tc && seg_mma_ok(a);
  const std::string nm =
      std::string(a.name ? a.name : "seg_gemm") + (tc ? (g_tc_bf16 ? "_tc_bf16" : "_tc") : a.f32 ? "_f32" : "_f64");
  const bool split = a.seg_ptr && a.vseg_ptr && a.nvseg > a.nseg && !g_no_alloc;
  static const bool trace = std::getenv("SGTN_TRACE_GEMM") != nullptr;
  if (trace)
    fprintf(stderr, "[gemm] %s nseg %d nterm %lld p %d q %d s %d splitk %d vseg %d\n", nm.c_str(), a.nseg,
            a.seg_ptr ? a.nterm : (long long)a.nseg, a.p, a.q, a.s, a.splitk, split ? a.nvseg : 0);
  KTimer t(nm.c_str(), st, fl);
  if (!split) {
    launch_seg(a, st, tc);
  } else {
    double* part = static_cast<double*>(
        stream_scratch(st, SC_SEG_PART, size_t(a.nvseg) * a.p * a.s * sizeof(double)));
    SegGemm b = a;
    b.seg_ptr = a.vseg_ptr;
    b.nseg = a.nvseg;
    b.out_by_seg = 1;
    b.O = part;
    b.os_i = a.s;
    b.os_j = 1;
    b.ors = (long long)a.p * a.s;
    b.alpha = 1.0;
    b.accumulate = 0;
    launch_seg(b, st, tc);
    long long total = (long long)a.nseg * a.p * a.s;
    int nb = int(std::min<long long>((total + 255) / 256, 148 * 16));
    seg_reduce_kernel<<<nb, 256, 0, st>>>(part, a.vfirst, a.nseg, a.p, a.s, a);
    ++g_count.launches;
  }
  g_count.flops += fl;
}

thread_local bool g_compute_f32 = false;
thread_local bool g_use_tc = false;
thread_local bool g_tc_bf16 = false;
thread_local bool g_no_alloc = false;

void gemm(const double* X, bool tx, long long ldx, const double* Y, bool ty, long long ldy, double* O, long long ldo,
          int m, int n, int k, double alpha, int accumulate, cudaStream_t st, int tri) {
  if (!tri && g_use_tc && g_compute_f32 && m >= 128 && n >= 64 && k >= 32 &&
      tc_gemm(X, tx, ldx, Y, ty, ldy, O, ldo, m, n, k, alpha, accumulate, st))
    return;
  SegGemm a;
  a.X = X;
  a.Y = Y;
  a.O = O;
  a.p = m;
  a.q = k;
  a.s = n;
  a.xs_i = tx ? 1 : ldx;
  a.xs_k = tx ? ldx : 1;
  a.ys_k = ty ? 1 : ldy;
  a.ys_j = ty ? ldy : 1;
  a.os_i = ldo;
  a.os_j = 1;
  a.nseg = 1;
  a.alpha = alpha;
  a.accumulate = accumulate;
  a.name = "gemm";
  a.tri = tri;
  // small outputs (Gram matrices, blocks of a Cholesky factor) take 16 x 32
  // tiles, so that more CTAs share the work and less of each tile is padding
  const bool small = (long long)m * n <= 160 * 160;
  const int bm = small ? 16 : m <= 16 ? 16 : m <= 32 ? 32 : 64, bn = small ? 32 : n <= 32 ? 32 : 64;
  a.tile_m = bm;
  a.tile_n = bn;
  long long tiles = (long long)((m + bm - 1) / bm) * ((n + bn - 1) / bn);
  if (tiles < 148 && k >= (small ? 64 : 256) && !g_no_alloc) {
    // few output tiles and a long reduction: split K over about two CTAs per
    // SM (chunks of at least 32), then reduce the partial products
    int nsplit = int(std::min<long long>((k + 31) / 32, std::max<long long>(2, (296 + tiles - 1) / tiles)));
    int chunk = ((k + nsplit - 1) / nsplit + TK - 1) / TK * TK;
    nsplit = (k + chunk - 1) / chunk;
    double* part =
        static_cast<double*>(stream_scratch(st, SC_SPLITK_PART, size_t(nsplit) * m * n * sizeof(double)));
    SegGemm b = a;
    b.O = part;
    b.os_i = n;
    b.os_j = 1;
    b.ors = (long long)m * n;
    b.nseg = nsplit;
    b.splitk = chunk;
    b.alpha = 1.0;
    b.accumulate = 0;
    b.name = "gemm_splitk";
    seg_gemm(b, st);
    splitk_reduce_kernel<<<blocks_for((long long)m * n), 256, 0, st>>>(part, nsplit, (long long)m * n, n, O, ldo, alpha,
                                                                        accumulate);
    ++g_count.launches;
    return;
  }
  seg_gemm(a, st);
}

void jacobi(double* X, int len, int p, long long si, long long sj, double* V, int max_sweeps, int* status,
            cudaStream_t st) {
  double tol = 1e-15 * sqrt(double(len > 1 ? len : 1));
  size_t smem = (size_t(len) * p + (V ? size_t(p) * p : 0)) * sizeof(double);
  const size_t kMaxSmem = 220 * 1024;
  // once per process (thread-safe initialisation of a local static): kernel
  // attributes, and the cluster size, up to 16 CTAs (one pair per warp and
  // step) if the device takes it
  static const int max_cluster = [kMaxSmem] {
    cudaFuncSetAttribute(jacobi_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxSmem));
    for (void* f : {(void*)jacobi_cluster_kernel<0>, (void*)jacobi_cluster_kernel<4>}) {
      cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxSmem));
    }
    int mc = 8;
    cudaLaunchConfig_t q = {};
    cudaLaunchAttribute qa[1];
    q.gridDim = dim3(16);
    q.blockDim = dim3(512);
    q.dynamicSmemBytes = 64 * 1024;
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = 16;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (void*)jacobi_cluster_kernel<0>, &q) == cudaSuccess && ncl >= 1)
      mc = 16;
    cudaGetLastError();
    return mc;
  }();
  const int npair = (p + 1) / 2;
  int P = std::max(1, std::min(max_cluster, npair));
  const int slots = (p + P - 1) / P;
  const size_t csmem = (size_t(slots) * len + (V ? size_t(slots) * p : 0) + size_t(slots)) * sizeof(double);
  const int nw = std::min(16, (npair + P - 1) / P);
  {
    KTimer t("jacobi_f64", st);
    if (p >= 8 && csmem <= kMaxSmem) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(P);
      cfg.blockDim = dim3(32 * nw);
      cfg.dynamicSmemBytes = csmem;
      cfg.stream = st;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = P;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (len <= 128)
        cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<4>, X, len, p, si, sj, V, max_sweeps, tol, status);
      else
        cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<0>, X, len, p, si, sj, V, max_sweeps, tol, status);
    } else if (smem <= kMaxSmem) {
      jacobi_smem_kernel<<<1, 1024, smem, st>>>(X, len, p, si, sj, V, max_sweeps, tol, status);
    } else {
      // flags (one per sweep) and the Frobenius norm live in the stream's scratch
      int* flags = static_cast<int*>(stream_scratch(st, SC_JAC_FLAGS, 256 * sizeof(int)));
      double* fro = static_cast<double*>(stream_scratch(st, SC_JAC_FRO, sizeof(double)));
      if (!flags || !fro) throw SgtnError(-3, "Jacobi scratch needs an allocation in an allocation-free call");
      cudaMemsetAsync(flags, 0, 256 * sizeof(int), st);
      int ms = max_sweeps > 256 ? 256 : max_sweeps;
      int nblk = ((p + 1) / 2 + 3) / 4;   // 4 warps (pairs) per CTA
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel, 128, 0);
      int dev = 0, nsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      int cap = per_sm * nsm;
      if (nblk > cap) nblk = cap;
      if (nblk < 1) nblk = 1;
      void* args[] = {&X, &len, &p, &si, &sj, &V, &ms, &tol, &status, &flags, &fro};
      cudaLaunchCooperativeKernel((void*)jacobi_coop_kernel, dim3(nblk), dim3(128), args, 0, st);
    }
  }
  ++g_count.launches;
}

namespace {
constexpr int kCholBlock = 48;   // blocks up to this size are factored by one CTA

void chol_base(double* W, int n, int ld, double shift, double* R, const double* Gd, int* status, int off,
               double* minratio, cudaStream_t st, bool f32) {
  static const bool attr = [] {
    cudaFuncSetAttribute(cholesky_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(cholesky_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    return true;
  }();
  (void)attr;
  if (f32)
    cholesky_inv_kernel<float><<<1, 1024, size_t(n) * (n + 2) * sizeof(float), st>>>(W, n, ld, shift, R, W, Gd,
                                                                                    status, off, minratio, off == 0);
  else
    cholesky_inv_kernel<double><<<1, 1024, size_t(n) * (n + 2) * sizeof(double), st>>>(W, n, ld, shift, R, W, Gd,
                                                                                      status, off, minratio, off == 0);
  ++g_count.launches;
}

// Recursive blocked Cholesky and inverse, in place: on entry W (n x n block,
// leading dimension ld) holds the upper triangle of G; on return R holds the
// factor of G + shift I and W its inverse.  With n = n1 + n2:
//   R11 = chol(G11), R12 = R11^{-T} G12, S = G22 - R12^T R12, R22 = chol(S),
//   R^{-1}_12 = -R11^{-1} R12 R22^{-1};
// the off-diagonal products are GEMMs over many CTAs, only the diagonal
// blocks of at most kCholBlock rows are factored by one CTA.
void chol_rec(double* W, int n, int ld, double shift, double* R, const double* Gd, int* status, int off,
              double* minratio, double* T, cudaStream_t st, bool f32) {
  if (n <= kCholBlock) {
    chol_base(W, n, ld, shift, R, Gd, status, off, minratio, st, f32);
    return;
  }
  const int n1 = std::min(n - 16, (n / 2 + 15) / 16 * 16), n2 = n - n1;
  double *W12 = W + n1, *W21 = W + (long long)n1 * ld, *W22 = W21 + n1;
  double *R12 = R + n1, *R21 = R + (long long)n1 * ld, *R22 = R21 + n1;
  chol_rec(W, n1, ld, shift, R, Gd, status, off, minratio, T, st, f32);
  gemm(W, true, ld, W12, false, ld, R12, ld, n1, n2, n1, 1.0, 0, st);        // R12 = R11^{-T} G12
  gemm(R12, true, ld, R12, false, ld, W22, ld, n2, n2, n1, -1.0, 1, st);     // W22 = G22 - R12^T R12
  chol_rec(W22, n2, ld, shift, R22, Gd + (long long)n1 * (ld + 1), status, off + n1, minratio, T, st, f32);
  gemm(R12, false, ld, W22, false, ld, T, n2, n1, n2, n2, 1.0, 0, st, 2);     // T = R12 R22^{-1}
  gemm(W, false, ld, T, false, n2, W12, ld, n1, n2, n1, -1.0, 0, st);         // (R^{-1})_12 = -R11^{-1} T
  const long long nz = (long long)n2 * n1;
  zero_blocks2_kernel<<<blocks_for(nz), 256, 0, st>>>(W21, R21, n2, n1, ld);
  ++g_count.launches;
}
}  // namespace

void cholesky_inv(const double* G, int n, double shift, double* R, double* Rinv, int* status, cudaStream_t st,
                  bool f32, double* minratio) {
  const double fl = double(n) * n * n;   // n^3/3 FMA factor + n^3/6 FMA inverse, 2 flop each
  KTimer t(f32 ? "cholesky_f32" : "cholesky_f64", st, fl);
  // the off-diagonal GEMMs run in FP64 whatever the caller's contraction precision
  const bool sf = g_compute_f32, su = g_use_tc;
  g_compute_f32 = g_use_tc = false;
  double* T = static_cast<double*>(stream_scratch(st, SC_CHOL_T, size_t(n) * n * sizeof(double)));
  if (!T) throw SgtnError(-3, "Cholesky scratch needs an allocation in an allocation-free call");
  // status and minratio are set by the first diagonal block (offset 0), which
  // runs before every other block of this factorisation in stream order
  if (Rinv != G) cudaMemcpyAsync(Rinv, G, size_t(n) * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  chol_rec(Rinv, n, n, shift, R, G, status, 0, minratio, T, st, f32);
  g_compute_f32 = sf;
  g_use_tc = su;
}

void gram_stats(const double* G, int k, double* out, cudaStream_t st) {
  gram_stats_kernel<<<1, 1024, 0, st>>>(G, k, out);
  ++g_count.launches;
}

void pchol_inv(const double* G, int n, double tol_rel, double tol_abs, double* R, double* Rinv, int32_t* perm,
               int* rank, cudaStream_t st) {
  static const bool attr = [] {
    cudaFuncSetAttribute(pchol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    return true;
  }();
  (void)attr;
  KTimer t("pcholesky_f64", st);
  pchol_inv_kernel<<<1, 1024, size_t(n) * n * sizeof(double), st>>>(G, n, tol_rel, tol_abs, R, Rinv, perm, rank);
  ++g_count.launches;
}

void vec_norms(const double* X, int len, int p, long long si, long long sj, double* out, cudaStream_t st) {
  if (p > 0) vec_norms_kernel<<<p, 256, 0, st>>>(X, len, p, si, sj, out);
  ++g_count.launches;
}

void gather_vecs(const double* X, int len, long long si, long long sj, const int32_t* perm, const double* scale, int k,
                 double* out, long long oi, long long oj, cudaStream_t st) {
  gather_vecs_kernel<<<blocks_for((long long)len * k), 256, 0, st>>>(X, len, si, sj, perm, scale, k, out, oi, oj);
  ++g_count.launches;
}

void permute3(const double* in, int A, int B, int Cd, double* out, cudaStream_t st) {
  permute3_kernel<<<blocks_for((long long)A * B * Cd), 256, 0, st>>>(in, A, B, Cd, out);
  ++g_count.launches;
}

void permute_nd(const double* in, int nd, const int* dims, const int* perm, double* out, cudaStream_t st) {
  PermArgs pa;
  pa.nd = nd;
  long long stride[6];
  long long s = 1;
  for (int k = nd - 1; k >= 0; --k) {
    stride[k] = s;
    s *= dims[k];
  }
  for (int k = 0; k < nd; ++k) {
    pa.in_stride[k] = stride[perm[k]];
    pa.out_dim[k] = dims[perm[k]];
  }
  permute_nd_kernel<<<blocks_for(s), 256, 0, st>>>(in, out, s, pa);
  ++g_count.launches;
}

void scatter_blocks(const double* blocks, int nseg, int chl, int kp, const int32_t* seg_bl, const int32_t* seg_u,
                    double* dense, long long n, cudaStream_t st) {
  long long total = (long long)nseg * chl * kp;
  scatter_blocks_kernel<<<blocks_for(total), 256, 0, st>>>(blocks, total, chl, kp, seg_bl, seg_u, dense, n);
  ++g_count.launches;
}

void fro_norm(const double* x, long long n, double* out, cudaStream_t st) { fro_norm_kernel<<<1, 1024, 0, st>>>(x, n, out);
  ++g_count.launches; }

void scale_by_inv(double* x, long long n, const double* norm, cudaStream_t st) {
  scale_by_inv_kernel<<<blocks_for(n), 256, 0, st>>>(x, n, norm);
  ++g_count.launches;
}

void pseudo_random(double* x, long long n, unsigned long long seed, cudaStream_t st) {
  pseudo_random_kernel<<<blocks_for(n), 256, 0, st>>>(x, n, seed);
  ++g_count.launches;
}

namespace {
// S = (3 I - G) / 2 from the upper triangle of a symmetric G (k x k)
__global__ void polar_factor_kernel(const double* G, int k, double* S) {
  const long long n = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = int(e / k), j = int(e % k);
    const double g = i <= j ? G[(long long)i * k + j] : G[(long long)j * k + i];
    S[e] = (i == j ? 1.5 : 0.0) - 0.5 * g;
  }
}
}  // namespace

void polar_factor(const double* G, int k, double* S, cudaStream_t st) {
  polar_factor_kernel<<<blocks_for((long long)k * k), 256, 0, st>>>(G, k, S);
  ++g_count.launches;
}

void add_cols(double* R, const double* Q, int rows, int k, int ldq, cudaStream_t st) {
  add_cols_kernel<<<blocks_for((long long)rows * k), 256, 0, st>>>(R, Q, rows, k, ldq);
  ++g_count.launches;
}

void scale_pow2(double* x, long long n, int e, cudaStream_t st) {
  scale_pow2_kernel<<<blocks_for(n), 256, 0, st>>>(x, n, e);
  ++g_count.launches;
}

void fill(double* x, long long n, double v, cudaStream_t st) { fill_kernel<<<blocks_for(n), 256, 0, st>>>(x, n, v);
  ++g_count.launches; }

void copy(double* dst, const double* src, long long n, cudaStream_t st) {
  copy_kernel<<<blocks_for(n), 256, 0, st>>>(dst, src, n);
  ++g_count.launches;
}

void boltzmann(const int64_t* E, long long n, int64_t Emin, double bd, double* out, cudaStream_t st) {
  boltzmann_kernel<<<blocks_for(n), 256, 0, st>>>(E, n, Emin, bd, out);
  ++g_count.launches;
}

void build_Wa(double* Wa, int nPd, int nE, int nG, int nSig, const int32_t* s_pu, const int32_t* s_pul,
              const int32_t* s_pur, const double* Bv, int bv_nb, const double* Bdl, int bdl_nb, cudaStream_t st) {
  long long n = (long long)nPd * nE * nG * nSig;
  build_Wa_kernel<<<blocks_for(n), 256, 0, st>>>(Wa, nPd, nE, nG, nSig, s_pu, s_pul, s_pur, Bv, bv_nb, Bdl, bdl_nb);
  ++g_count.launches;
}

void build_Wk(double* Wk, int nPr, int nE, int nPdr, int nLR, int nGR, const int32_t* l_pl, const int32_t* l_pdl,
              const double* Bh, int bh_nb, const double* Bdr, int bdr_nb, cudaStream_t st) {
  long long n = (long long)nPr * nE * nPdr * nLR * nGR;
  build_Wk_kernel<<<blocks_for(n), 256, 0, st>>>(Wk, nPr, nE, nPdr, nLR, nGR, l_pl, l_pdl, Bh, bh_nb, Bdr, bdr_nb);
  ++g_count.launches;
}

}  // namespace sgtn
