// Host wrappers of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <stdexcept>
#include <string>

// The library's error: a status code of include/sgtn.h and a message.
struct SgtnError : std::runtime_error {
  int code;
  SgtnError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

namespace sgtn {

// A double that several host threads add to.
struct AtomicSum {
  std::atomic<double> v{0.0};
  void operator+=(double x) {
    double o = v.load(std::memory_order_relaxed);
    while (!v.compare_exchange_weak(o, o + x, std::memory_order_relaxed)) {
    }
  }
  operator double() const { return v.load(std::memory_order_relaxed); }
};
// Process-wide diagnostics: kernel launches issued by this library and the
// algorithmic floating-point operations of its contractions (summed over all
// host threads driving handles).
struct Counters {
  std::atomic<long long> launches{0};
  AtomicSum flops;
  std::atomic<long long> evals{0};
  std::atomic<long long> device_allocs{0};   // cudaMalloc calls made by the library
};
extern Counters g_count;
// Every device allocation of the library goes through here, so that the
// allocation-free entry point can be checked to make none.
template <class T>
inline cudaError_t lib_malloc(T** p, size_t bytes) {
  ++g_count.device_allocs;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
// The three mode flags below belong to the calling host thread: a handle's
// call sets them for its own duration, so handles driven by different threads
// (one stream each) do not see each other's modes.
// When set, every contraction (seg_gemm / gemm) multiplies and accumulates in
// FP32; the SVDs, norms and log-norms stay FP64.  Set per call from the handle.
extern thread_local bool g_compute_f32;
// When set (with g_compute_f32), dense GEMMs large enough for 128 x 128 tiles
// run on tcgen05 tensor cores (3xTF32).
extern thread_local bool g_use_tc;
// When set (with g_use_tc), the segmented tensor-core contractions split
// their operands into three BF16 slices (kind::f16 MMAs) instead of two TF32
// parts; dense GEMMs stay 3xTF32.
extern thread_local bool g_tc_bf16;
// When set, the GEMM helpers allocate no device memory of their own (no
// split-K or split-segment partial buffers): set by the allocation-free entry
// point for the duration of its call.
extern thread_local bool g_no_alloc;

// Device scratch private to one stream: slot `slot` of stream `st`, at least
// `bytes` long, reused by every later call on that stream (stream order keeps
// the uses apart).  Growing it waits for the stream.  nullptr if it would have
// to grow while g_no_alloc is set.
enum ScratchSlot { SC_SEG_PART, SC_SPLITK_PART, SC_CHOL_T, SC_JAC_FLAGS, SC_JAC_FRO, SC_TC_BUF, SC_KPART, SC_NSLOT };
void* stream_scratch(cudaStream_t st, int slot, size_t bytes);
void stream_scratch_release(cudaStream_t st);

// Optional per-kernel timing with CUDA events on the launching stream.
// KTimer brackets one launch; pairs are resolved when read.
void ktimer_begin(const char* name, cudaStream_t st);
void ktimer_end(cudaStream_t st, double flops);
void ktimer_enable(bool on);
void ktimer_add_flops(const char* name, double flops);   // work known only after the launch
void ktimer_reset();
bool ktimer_read(const char* name, double* ms, long long* n, double* flops);
std::string ktimer_names();   // comma-separated names seen so far
struct KTimer {
  cudaStream_t st;
  double flops;
  KTimer(const char* name, cudaStream_t s, double f = 0.0) : st(s), flops(f) { ktimer_begin(name, s); }
  ~KTimer() { ktimer_end(st, flops); }
};

// Segmented gathered GEMM, double precision:
//   O[seg] (+)= alpha * sum_{t in seg} coef[cidx[t]] * X_t * (Y_t diag(cs[csrow[t]]))
// Blocks: X_t is p x q, Y_t is q x s, O_seg is p x s, addressed with element
// strides (xs_i, xs_k), (ys_k, ys_j), (os_i, os_j) from block offsets
//   xoff = xr*xrs + xc*xcs, yoff = yr*yrs + yc*ycs, ooff = or*ors + oc*ocs.
// Table mode when seg_ptr != nullptr; otherwise uniform batch mode: segment b
// has a single term with xr = yr = or = b and xc = yc = oc = 0, coefficient 1.
struct SegGemm {
  const double* X = nullptr;
  const double* Y = nullptr;
  double* O = nullptr;
  int p = 0, q = 0, s = 0;
  long long xs_i = 0, xs_k = 0, ys_k = 0, ys_j = 0, os_i = 0, os_j = 0;
  long long xrs = 0, xcs = 0, yrs = 0, ycs = 0, ors = 0, ocs = 0;
  const int32_t *seg_ptr = nullptr, *seg_or = nullptr, *seg_oc = nullptr;
  const int32_t *xr = nullptr, *xc = nullptr, *yr = nullptr, *yc = nullptr, *cidx = nullptr, *csrow = nullptr;
  const double* coef = nullptr;
  const double* cs = nullptr;
  long long cs_ld = 0;
  int nseg = 1;
  int out_by_seg = 0;    // table mode: output block offset = segment index * ors
  int f32 = 0;           // multiply-accumulate in FP32 (inputs and outputs stay FP64)
  int splitk = 0;        // uniform mode: segment t sums k in [t*splitk, (t+1)*splitk) of one product
  long long nterm = 0;   // host-side term count for the FLOP counter (table mode)
  double alpha = 1.0;
  int accumulate = 0;
  const char* name = nullptr;   // timing label (role of the call); "_f32" / "_f64" is appended
  int tile_m = 0, tile_n = 0;   // CTA tile (16/32/64 x 32/64); 0: from the block shape
  // uniform mode, structure of one product: tri & 1 -- only the upper triangle
  // of the (square) output is needed (tiles wholly below the diagonal are
  // skipped and left unwritten); tri & 2 -- Y is upper triangular (the
  // reduction of output column j stops at k = j)
  int tri = 0;
  // optional balanced split of long segments (table mode): the virtual
  // segments are multiplied into a scratch block each and summed per segment
  // in a fixed order (deterministic)
  const int32_t *vseg_ptr = nullptr, *vfirst = nullptr;
  int nvseg = 0;
  // set by the launcher, not by callers: each segment's (term, k-chunk)
  // sequence is cut into kpart contiguous parts, one CTA each, whose partial
  // blocks are summed in part order afterwards (small grids fill the GPU)
  int kpart = 1;
  // table mode, optional: rows of X (blocks xr * (xrs / xs_i) + i) and of Y
  // (yr * (yrs / ys_k) + k) that exist in memory.  When set, a TF32-mode call
  // with row-major blocks may run on the tensor cores (seg_mma), whose tile
  // copies are bounded by these extents.
  long long x_rows = 0, y_rows = 0;
};
void seg_gemm(const SegGemm& a, cudaStream_t st);
// Tensor-core form of seg_gemm (3xTF32 on tcgen05): whether a call can take
// it, and the launch (false if nothing was launched).
bool seg_mma_ok(const SegGemm& a);
bool seg_mma(const SegGemm& a, cudaStream_t st);

// Plain row-major GEMM helper on top of seg_gemm: O[m x n] = alpha * op(X) op(Y)
void gemm(const double* X, bool tx, long long ldx, const double* Y, bool ty, long long ldy, double* O,
          long long ldo, int m, int n, int k, double alpha, int accumulate, cudaStream_t st, int tri = 0);
// G (n x n) = X^T X for X (m x n, leading dimension ldx): upper triangle only
// out[0] = max |G_ij - delta_ij| over the upper triangle (NaN if any entry is
// not finite), out[1] = trace of G (k x k); device outputs
void gram_stats(const double* G, int k, double* out, cudaStream_t st);
inline void gram_upper(const double* X, long long ldx, double* G, int n, int m, cudaStream_t st) {
  gemm(X, true, ldx, X, false, ldx, G, n, n, n, m, 1.0, 0, st, 1);
}

// One-sided Jacobi (Hestenes) on the p vectors of a matrix: vector j has
// element i at X[i*si + j*sj], i < len.  On return the vectors are mutually
// orthogonal; V (p x p, column j at V[j*p], may be null) accumulates the
// rotations.  status[0] = sweeps used, or -1 if max_sweeps ran out.
void jacobi(double* X, int len, int p, long long si, long long sj, double* V, int max_sweeps, int* status,
            cudaStream_t st);
// Upper Cholesky factor R of (G + shift I) (n x n, row-major; R^T R = G + shift I)
// and R^{-1}, one CTA.  status[0] = 0 on success, j+1 if pivot j was not positive.
// f32: factor in FP32 arithmetic (inputs and outputs stay FP64).  minratio
// (optional): smallest pivot over the matching diagonal entry of G + shift I,
// i.e. how much of a column survived the elimination (1: orthogonal columns).
void cholesky_inv(const double* G, int n, double shift, double* R, double* Rinv, int* status, cudaStream_t st,
                  bool f32 = false, double* minratio = nullptr);
// Cholesky with diagonal pivoting of a PSD G (n x n, n <= 160), stopped at the
// numerical rank (largest remaining pivot <= max(tol_rel * max diag G, tol_abs)):
// rank[0] = r, perm[0..r) the pivot order, R and R^{-1} (r x r upper triangular,
// leading dimension n) with G[perm][perm] = R^T R on the leading block.  One CTA.
void pchol_inv(const double* G, int n, double tol_rel, double tol_abs, double* R, double* Rinv, int32_t* perm,
               int* rank, cudaStream_t st);
double* trace_scratch();
void vec_norms(const double* X, int len, int p, long long si, long long sj, double* out, cudaStream_t st);
// out[i*oi + jj*oj] = scale[jj] * X[i*si + perm[jj]*sj]
void gather_vecs(const double* X, int len, long long si, long long sj, const int32_t* perm, const double* scale,
                 int k, double* out, long long oi, long long oj, cudaStream_t st);
// C[m x n] (+)= alpha op(X) op(Y) on tcgen05 tensor cores with 3xTF32 splitting
// (about FP32 accuracy); false if it could not be launched.
bool tc_gemm(const double* X, bool tx, long long ldx, const double* Y, bool ty, long long ldy, double* C, long long ldc,
             int m, int n, int k, double alpha, int accumulate, cudaStream_t st);
int tc_gemm_take_error(cudaStream_t st);
// deterministic pseudo-random numbers in [-1, 1] (SplitMix64 of seed + index)
void pseudo_random(double* x, long long n, unsigned long long seed, cudaStream_t st);
// S = (3 I - G) / 2 (k x k) from the upper triangle of a symmetric G: for a
// Gram matrix G = Q^T Q = I + E of nearly orthonormal vectors, Q S is
// orthonormal to O(|E|^2) (first step of the Newton iteration for the polar
// factor) and spans the same space
void polar_factor(const double* G, int k, double* S, cudaStream_t st);
// R[i][j] += Q[i*ldq + j] for j < k  (R is rows x k, Q is rows x ldq)
void add_cols(double* R, const double* Q, int rows, int k, int ldq, cudaStream_t st);
// generic permutation of an nd-array (nd <= 6): out axis k = in axis perm[k]
void permute_nd(const double* in, int nd, const int* dims, const int* perm, double* out, cudaStream_t st);
// dense[(bl*chl + i)*n + u*kp + j] = blocks[seg][i][j] for seg's (bl, u)
void scatter_blocks(const double* blocks, int nseg, int chl, int kp, const int32_t* seg_bl, const int32_t* seg_u,
                    double* dense, long long n, cudaStream_t st);
// out[b][a][c] = in[a][b][c]
void permute3(const double* in, int A, int B, int Cd, double* out, cudaStream_t st);
// Frobenius norm (deterministic), result on device in *out
void fro_norm(const double* x, long long n, double* out, cudaStream_t st);
void scale_by_inv(double* x, long long n, const double* norm, cudaStream_t st);
// x *= 2^-e (exact in binary floating point)
void scale_pow2(double* x, long long n, int e, cudaStream_t st);
void fill(double* x, long long n, double v, cudaStream_t st);
void copy(double* dst, const double* src, long long n, cudaStream_t st);

// exp(-beta (E - Emin) / denom)
void boltzmann(const int64_t* E, long long n, int64_t Emin, double beta_over_denom, double* out, cudaStream_t st);
// dense weight matrices of a column (see boundary.cu)
void build_Wa(double* Wa, int nPd, int nE, int nG, int nSig, const int32_t* s_pu, const int32_t* s_pul,
              const int32_t* s_pur, const double* Bv, int bv_nb, const double* Bdl, int bdl_nb, cudaStream_t st);
void build_Wk(double* Wk, int nPr, int nE, int nPdr, int nLR, int nGR, const int32_t* l_pl, const int32_t* l_pdl,
              const double* Bh, int bh_nb, const double* Bdr, int bdr_nb, cudaStream_t st);

}  // namespace sgtn
