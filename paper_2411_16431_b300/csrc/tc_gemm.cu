// Tensor-core GEMM for sm_103a: C (M x N, FP64 out) = A (M x K) * B (K x N)
// with 3xTF32 splitting (Ootomo & Yokota 2022): each operand X = X_hi + X_lo
// with X_hi = tf32(X), X_lo = tf32(X - X_hi); C = A_hi B_hi + A_hi B_lo +
// A_lo B_hi accumulated in FP32 in tensor memory, which keeps about FP32
// accuracy while running on the 5th-generation tensor cores.
//
// One CTA computes a 128 x 128 tile: operand tiles of 128 rows x 32 TF32
// (128 bytes, 128B-swizzled) arrive by TMA into a 3-stage shared-memory ring
// guarded by mbarriers; one thread issues tcgen05.mma (kind::tf32, M=128,
// N=128, K=8) into a TMEM accumulator; all four warps read it back with
// tcgen05.ld.  Every wait is bounded: on time-out the CTA records an error
// and skips its work, and it always frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "convert.h"
#include "kern.h"

namespace sgtn {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 4;                 // 16 KB, same for A and B tiles
constexpr int STAGE_BYTES = 4 * TILE_BYTES;             // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024; // + alignment slack
constexpr long long SPIN_LIMIT = 1ll << 26;

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait on the given phase parity; returns false on time-out
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ inline uint64_t smem_desc(const void* p) {
  uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;          // start address
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, A/B TF32 K-major, D FP32, M = 128, N = 128
constexpr uint32_t IDESC = (1u << 4)                 // D format F32
                           | (2u << 7)               // A format TF32
                           | (2u << 10)              // B format TF32
                           | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ inline void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(128, 1)
    tc_gemm_3xtf32_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                          const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, int M,
                          int N, int K, double* C, long long ldc, double alpha, int accumulate, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int ktiles = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kt = 0; kt < ktiles; ++kt) {
      int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (abort_flag) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(st + 0 * TILE_BYTES, &mAhi, &full[s], kt * BK, m0);
      tma_load_2d(st + 1 * TILE_BYTES, &mAlo, &full[s], kt * BK, m0);
      tma_load_2d(st + 2 * TILE_BYTES, &mBhi, &full[s], kt * BK, n0);
      tma_load_2d(st + 3 * TILE_BYTES, &mBlo, &full[s], kt * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      int s = kt % STAGES;
      if (!mbar_wait(&full[s], (kt / STAGES) & 1)) {
        atomicExch(&abort_flag, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = smem + s * STAGE_BYTES;
      for (int kk = 0; kk < BK / 8; ++kk) {
        uint64_t ahi = smem_desc(st + 0 * TILE_BYTES) + (uint64_t)(kk * 32 >> 4);
        uint64_t alo = smem_desc(st + 1 * TILE_BYTES) + (uint64_t)(kk * 32 >> 4);
        uint64_t bhi = smem_desc(st + 2 * TILE_BYTES) + (uint64_t)(kk * 32 >> 4);
        uint64_t blo = smem_desc(st + 3 * TILE_BYTES) + (uint64_t)(kk * 32 >> 4);
        uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, ahi, bhi, acc);
        mma_tf32(tmem, ahi, blo, 1u);
        mma_tf32(tmem, alo, bhi, 1u);
      }
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(&done_bar);
    else atomicExch(&abort_flag, 1);
  }
  __syncwarp();
  // epilogue: all 4 warps, warp w owns TMEM lanes / tile rows 32w..32w+31
  bool have = !abort_flag && mbar_wait(&done_bar, 0);
  __syncthreads();
  if (have && !abort_flag) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
          "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
            "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
            "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        for (int j = 0; j < 32; ++j) {
          int col = n0 + c0 + j;
          if (col < N) {
            double v = alpha * (double)__uint_as_float(r[j]);
            double* o = C + (long long)row * ldc + col;
            *o = accumulate ? *o + v : v;
          }
        }
      }
    }
  }
  if (threadIdx.x == 0 && (abort_flag || !have)) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
}

// X_hi / X_lo (rows x kpad, fp32, zero padded) from a strided FP64 operand:
// element (i, k) at X[i * si + k * sk]
__global__ void split_tf32_kernel(const double* X, long long si, long long sk, int rows, int K, int kpad, float* hi,
                                  float* lo) {
  long long n = (long long)rows * kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int i = int(e / kpad), k = int(e % kpad);
    float h = 0.f, l = 0.f;
    if (k < K) {
      double v = X[i * si + k * sk];
      // round to TF32 (10 mantissa bits) with round-to-nearest on the dropped bits
      uint32_t b = __float_as_uint((float)v);
      b = (b + 0x1000u) & 0xFFFFE000u;
      h = __uint_as_float(b);
      float rem = (float)(v - (double)h);
      uint32_t c = __float_as_uint(rem);
      c = (c + 0x1000u) & 0xFFFFE000u;
      l = __uint_as_float(c);
    }
    hi[e] = h;
    lo[e] = l;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap* map, const float* base, int rows, int kpad) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 4};
  cuuint32_t box[2] = {BK, BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

// Error flag of the tensor-core kernels (a wait that ran out of iterations):
// one static device word per device, shared by all streams (it only goes
// 0 -> 1 on the device), so that no call ever allocates for it.
static __device__ int g_tc_err;
static int* tc_err_flag() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tc_err) != cudaSuccess) return nullptr;
  return static_cast<int*>(p);
}

// C[m x n] (+)= alpha * op(X) op(Y), operands FP64 in memory, 3xTF32 tensor cores.
// Returns false (nothing launched) if the tensor map cannot be built.
bool tc_gemm(const double* X, bool tx, long long ldx, const double* Y, bool ty, long long ldy, double* C, long long ldc,
             int m, int n, int k, double alpha, int accumulate, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0) return true;
  int kpad = (k + 3) / 4 * 4;   // 16-byte row pitch for TMA
  int* const err = tc_err_flag();
  if (!err) return false;
  size_t need = 2 * (size_t(m) + n) * kpad;
  float* buf = static_cast<float*>(stream_scratch(st, SC_TC_BUF, need * sizeof(float)));
  if (!buf) return false;   // would allocate in an allocation-free call: the SIMT path allocates nothing
  float* ahi = buf;
  float* alo = ahi + size_t(m) * kpad;
  float* bhi = alo + size_t(m) * kpad;
  float* blo = bhi + size_t(n) * kpad;
  // A: element (i, kk) of op(X); B^T: element (j, kk) of op(Y)^T
  long long xsi = tx ? 1 : ldx, xsk = tx ? ldx : 1;
  long long ysj = ty ? ldy : 1, ysk = ty ? 1 : ldy;
  auto blocks = [](long long e) { return int(std::min<long long>((e + 255) / 256, 148ll * 16)); };
  split_tf32_kernel<<<blocks((long long)m * kpad), 256, 0, st>>>(X, xsi, xsk, m, k, kpad, ahi, alo);
  split_tf32_kernel<<<blocks((long long)n * kpad), 256, 0, st>>>(Y, ysj, ysk, n, k, kpad, bhi, blo);
  g_count.launches += 2;
  CUtensorMap mA1, mA2, mB1, mB2;
  if (!make_map(&mA1, ahi, m, kpad) || !make_map(&mA2, alo, m, kpad) || !make_map(&mB1, bhi, n, kpad) ||
      !make_map(&mB2, blo, n, kpad))
    return false;
  static const bool attr = [] {
    cudaFuncSetAttribute(tc_gemm_3xtf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    return true;
  }();
  (void)attr;
  dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM);
  double fl = 2.0 * m * n * k;
  {
    KTimer t("tc_gemm_3xtf32", st, fl);
    tc_gemm_3xtf32_kernel<<<grid, 128, SMEM_BYTES, st>>>(mA1, mA2, mB1, mB2, m, n, k, C, ldc, alpha, accumulate, err);
  }
  ++g_count.launches;
  g_count.flops += fl;
  return true;
}



// ---------------------------------------------------------------------------
// Segmented gathered GEMM on the tensor cores (the TF32-mode form of seg_gemm
// for row-major blocks):  O[seg] (+)= alpha * sum_{t in seg} coef_t X_t Y_t,
// X_t a p x q block (row pitch xs_i), Y_t a q x s block (row pitch ys_k).
// This is the sparse site diagram of Fig. 7(b) -- a sum over cluster states of
// chi x chi products of gathered MPS and environment blocks, each weighted by
// the state's Boltzmann factor -- and the environment updates built the same
// way.  Persistent CTAs (one per SM) walk their share of the work items
// (segment, 128-row tile, BN-column tile) and, inside an item, the flattened
// (term, 32-wide k-chunk) sequence:
//   warp 0: TMA copies of the FP64 X tile (p rows, at most 128, x 32) and Y
//     tile (32 x BN) of the next chunk into a 3- to 6-stage shared-memory ring (the
//     lanes fetch the term indices and coefficients of 32 items at a time);
//   warps 4-11: each chunk's FP64 tiles are converted to FP32 on their bit
//     patterns (B300 runs FP64 instructions, conversions included, at a small
//     fraction of its FP32 and integer rates), scaled (Y by the term's
//     coefficient, rows k >= q zeroed), split into TF32 high and low parts and
//     written back in place in the 128-byte-swizzled K-major layout the MMA
//     reads (the FP64 tile and its two TF32 halves take the same bytes);
//   warp 1 (one lane): 3 x 4 tcgen05.mma kind::tf32 (hi*hi + hi*lo + lo*hi)
//     per chunk into one of four TMEM accumulators (128 lanes x BN columns);
//   warps 12-15: when an item's last chunk is multiplied, its accumulator is
//     read with tcgen05.ld and written (or added) to O in FP64, while the MMAs
//     of the next items go to the other accumulators.
// Every wait is bounded: on a time-out the CTA records the error, stops, waits
// (bounded) for its own copies and MMAs in flight and frees its tensor memory.
namespace {

constexpr int SG_BM = 128, SG_BK = 32, SG_NACC = 4, SG_MAXST = 6;
constexpr int SG_A_BYTES = SG_BM * SG_BK * 8;                 // FP64 X tile = TF32 hi + lo
// a stage holds the X tile and a 32 x BN FP64 Y tile; as many stages as fit
// in 216 KB (3 for BN = 128 up to 6 for BN = 16)
template <int BN>
struct SgRing {
  static constexpr int kStageBytes = SG_A_BYTES + BN * SG_BK * 8;
  static constexpr int kStages = (216 * 1024 / kStageBytes) < SG_MAXST ? (216 * 1024 / kStageBytes) : SG_MAXST;
  static constexpr int kSmem = kStages * kStageBytes + 1024;
};
constexpr int SG_NCONV = 8;                                  // converter warps
constexpr int SG_THREADS = 32 * (4 + SG_NCONV + 4);

struct SegMmaArgs {
  const int32_t *seg_ptr, *seg_or, *seg_oc, *xr, *yr, *cidx;
  const double* coef;
  long long xrow_unit, yrow_unit;   // tensor rows per unit of xr / yr
  int p, q, s, nseg, ntm, ntn, out_by_seg, accumulate;
  int bmx;   // rows of an X tile copied: p rounded up to 8, at most 128
  long long ors, ocs, os_i;
  double* O;
  double alpha;
  int* err;
};

__device__ inline bool sg_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const uint32_t addr = smem_u32(bar);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  return false;
}
// D (+)= A B, kind::tf32, instruction descriptor idesc; accumulate = 0 starts D afresh
__device__ inline void sg_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// byte offset of 4 consecutive TF32 (k = 4 c .. 4 c + 3) of row r in a
// 128-byte-swizzled K-major tile whose base is 1024-byte aligned
__device__ inline uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }
// D (+)= A B, kind::f16 with BF16 operands
__device__ inline void sg_mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// three BF16 slices of an FP32 value, f = hi + mid + lo up to the last 24
// bits (round to nearest at each slice; the remainders are exact in FP32)
__device__ inline void sg_split_bf16x3(float f, uint16_t& h, uint16_t& m, uint16_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(f);
  const float r1 = f - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}
// 4 consecutive k (chunk c of 4, k = 4c .. 4c+3) of row r as BF16 slices in
// 128-byte-swizzled K-major tiles: the high slice in bytes 0-63 of the row
// of tile t0, the middle slice in bytes 64-127, the low slice in bytes 0-63
// of tile t1
__device__ inline void sg_store_bf16x3(unsigned char* t0, unsigned char* t1, int r, int c, float4 v) {
  uint16_t h[4], m[4], l[4];
  sg_split_bf16x3(v.x, h[0], m[0], l[0]);
  sg_split_bf16x3(v.y, h[1], m[1], l[1]);
  sg_split_bf16x3(v.z, h[2], m[2], l[2]);
  sg_split_bf16x3(v.w, h[3], m[3], l[3]);
  auto pack = [](const uint16_t* x) {
    return make_uint2((uint32_t)x[0] | ((uint32_t)x[1] << 16), (uint32_t)x[2] | ((uint32_t)x[3] << 16));
  };
  const uint32_t in16 = 8u * (uint32_t)(c & 1);   // byte offset inside the 16-byte chunk
  *reinterpret_cast<uint2*>(t0 + sw128(r, c >> 1) + in16) = pack(h);
  *reinterpret_cast<uint2*>(t0 + sw128(r, 4 + (c >> 1)) + in16) = pack(m);
  *reinterpret_cast<uint2*>(t1 + sw128(r, c >> 1) + in16) = pack(l);
}
__device__ inline void sg_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// split an FP32 value into TF32 parts (10 mantissa bits, nearest on the
// dropped bits): the high part and the TF32 rounding of the exact remainder,
// in FP32 and integer arithmetic only
__device__ inline float sg_cvt(double v) { return f64_to_f32_int(v); }
__device__ inline void sg_split(float f, float& hi, float& lo) {
  const uint32_t b = (__float_as_uint(f) + 0x1000u) & 0xFFFFE000u;
  hi = __uint_as_float(b);
  lo = __uint_as_float((__float_as_uint(f - hi) + 0x1000u) & 0xFFFFE000u);
}

// What the producer tells the other roles about the chunk in a stage: the
// term's coefficient, the chunk's k offset, and whether it opens or closes a
// work item (or, with SG_STOP, that no chunk follows).
constexpr int SG_FIRST = 1, SG_LAST = 2, SG_STOP = 4;
struct SgMeta {
  double cf;
  int kc, flags;
};

template <int BN, bool BF>
__global__ void __launch_bounds__(SG_THREADS, 1)
    seg_mma_3xtf32_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mY,
                          const __grid_constant__ SegMmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[SG_MAXST], conv[SG_MAXST], empty[SG_MAXST], accf[SG_NACC], acce[SG_NACC],
      fin;
  __shared__ SgMeta meta[SG_MAXST];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;
  __shared__ uint32_t issued[SG_MAXST];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_seg = a.ntm * a.ntn;
  const int nitems = a.nseg * per_seg;
  const int nk = (a.q + SG_BK - 1) / SG_BK;
  constexpr uint32_t B_BYTES = BN * SG_BK * 8;
  constexpr int SG_STAGES = SgRing<BN>::kStages, SG_STAGE_BYTES = SgRing<BN>::kStageBytes;
  constexpr uint32_t TMEM_COLS = 128 * SG_NACC;   // SG_NACC accumulators of up to 128 columns
  // kind::tf32 (operand format 2) or kind::f16 with BF16 operands (format 1); D in FP32
  constexpr uint32_t IDESC_SG = (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
                                ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(SG_BM >> 4) << 24);

  if (threadIdx.x == 0) {
    for (int s = 0; s < SG_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], SG_NCONV);
      mbar_init(&empty[s], 1);
      issued[s] = 0;
    }
    for (int b = 0; b < SG_NACC; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
    }
    mbar_init(&fin, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  volatile int* abt = &abort_flag;

  if (warp == 0) {
    // producer (whole warp): the lanes load the segment bounds and first-term
    // indices of 32 work items at once (most segments hold one term), lane 0
    // fills the ring
    uint32_t g = 0;
    bool run = true;
    const int G = gridDim.x;
    for (int base = blockIdx.x; base < nitems && run; base += 32 * G) {
      const int my = base + lane * G;
      int mt0 = 0, mt1 = 0, mxr = 0, myr = 0;
      double mcf = 1.0;
      if (my < nitems) {
        const int seg = my / per_seg;
        mt0 = a.seg_ptr[seg];
        mt1 = a.seg_ptr[seg + 1];
        if (mt1 > mt0) {
          mxr = a.xr[mt0];
          myr = a.yr[mt0];
          if (a.coef) mcf = a.coef[a.cidx[mt0]];
        }
      }
      for (int e = 0; e < 32 && run; ++e) {
        const int it = base + e * G;
        if (it >= nitems) break;
        const int r = it % per_seg;
        const int i0 = (r / a.ntn) * SG_BM, j0 = (r % a.ntn) * BN;
        const int t0 = __shfl_sync(0xffffffffu, mt0, e), t1 = __shfl_sync(0xffffffffu, mt1, e);
        int txr = __shfl_sync(0xffffffffu, mxr, e), tyr = __shfl_sync(0xffffffffu, myr, e);
        double cf = __shfl_sync(0xffffffffu, mcf, e);
        for (int t = t0; t < t1 && run; ++t) {
          if (t > t0) {   // further terms of a segment: one load per term
            txr = a.xr[t];
            tyr = a.yr[t];
            cf = a.coef ? a.coef[a.cidx[t]] : 1.0;
          }
          const int xrow = int((long long)txr * a.xrow_unit) + i0;
          const int yrow = int((long long)tyr * a.yrow_unit);
          for (int kc = 0; kc < nk; ++kc, ++g) {
            const int s = g % SG_STAGES;
            // lane 0 waits for the stage to drain; the verdict is the warp's
            int ok = 1;
            if (lane == 0 && g >= SG_STAGES) ok = sg_wait(&empty[s], ((g / SG_STAGES) - 1) & 1, abt);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
              if (lane == 0) atomicExch(&abort_flag, 1);
              run = false;
              break;
            }
            if (lane == 0) {
              meta[s].cf = cf;
              meta[s].kc = kc;
              meta[s].flags = (t == t0 && kc == 0 ? SG_FIRST : 0) | (t == t1 - 1 && kc == nk - 1 ? SG_LAST : 0);
              unsigned char* st = smem + s * SG_STAGE_BYTES;
              mbar_expect_tx(&full[s], a.bmx * (SG_BK * 8) + B_BYTES);
              tma_load_2d(st, &mX, &full[s], kc * SG_BK, xrow);
              tma_load_2d(st + SG_A_BYTES, &mY, &full[s], j0, yrow + kc * SG_BK);
              issued[s] += 1;
            }
            __syncwarp();
          }
        }
      }
    }
    // sentinel: a stage with no data whose meta says that no chunk follows
    if (run && lane == 0) {
      const int s = g % SG_STAGES;
      if (g >= SG_STAGES && !sg_wait(&empty[s], ((g / SG_STAGES) - 1) & 1, abt)) {
        atomicExch(&abort_flag, 1);
      } else {
        meta[s].flags = SG_STOP;
        sg_arrive(&full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: follows the chunks' meta; one accumulator per work item
      uint32_t g = 0, n = 0, buf = 0;
      for (;; ++g) {
        const int s = g % SG_STAGES;
        if (!sg_wait(&conv[s], (g / SG_STAGES) & 1, abt)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        const int fl = meta[s].flags;
        if (fl & SG_STOP) break;
        if (fl & SG_FIRST) {
          buf = n % SG_NACC;
          if (n >= SG_NACC && !sg_wait(&acce[buf], ((n / SG_NACC) - 1) & 1, abt)) {
            atomicExch(&abort_flag, 1);
            break;
          }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + buf * 128;
        unsigned char* st = smem + s * SG_STAGE_BYTES;
        const uint64_t ahi = smem_desc(st), alo = smem_desc(st + SG_A_BYTES / 2);
        const uint64_t bhi = smem_desc(st + SG_A_BYTES), blo = smem_desc(st + SG_A_BYTES + B_BYTES / 2);
        if constexpr (BF) {
          // each 128-byte row holds [high slice | middle slice] of the 32 k of the
          // chunk, the second tile the low slice: per 16-wide k step, the six
          // products of slices whose orders add up to at most 2 (about FP32 accuracy)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t o = (uint64_t)((kk * 32) >> 4), om = (uint64_t)((64 + kk * 32) >> 4);
            sg_mma_bf16(d, ahi + o, bhi + o, IDESC_SG, ((fl & SG_FIRST) && kk == 0) ? 0u : 1u);
            sg_mma_bf16(d, ahi + o, bhi + om, IDESC_SG, 1u);
            sg_mma_bf16(d, ahi + om, bhi + o, IDESC_SG, 1u);
            sg_mma_bf16(d, ahi + o, blo + o, IDESC_SG, 1u);
            sg_mma_bf16(d, alo + o, bhi + o, IDESC_SG, 1u);
            sg_mma_bf16(d, ahi + om, bhi + om, IDESC_SG, 1u);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < SG_BK / 8; ++kk) {
            const uint64_t o = (uint64_t)((kk * 32) >> 4);
            sg_mma(d, ahi + o, bhi + o, IDESC_SG, ((fl & SG_FIRST) && kk == 0) ? 0u : 1u);
            sg_mma(d, ahi + o, blo + o, IDESC_SG, 1u);
            sg_mma(d, alo + o, bhi + o, IDESC_SG, 1u);
          }
        }
        mma_commit(&empty[s]);
        if (fl & SG_LAST) {
          mma_commit(&accf[buf]);
          ++n;
        }
      }
      // every MMA this thread issued has completed before the memory is freed
      mma_commit(&fin);
      if (!mbar_wait(&fin, 0)) atomicExch(&abort_flag, 1);
    }
  } else if (warp >= 4 && warp < 4 + SG_NCONV) {
    // converters: FP64 tiles -> scaled TF32 hi / lo, in place, swizzled K-major.
    // Work units of 4 consecutive k (one 16-byte TF32 chunk): X units go
    // lane-fast along a row's 8 chunks (a warp reads 4 rows of 256 bytes and
    // writes 4 swizzled rows, no bank conflicts), Y units lane-fast along the
    // columns j (contiguous reads); rows of X at or past bmx were not copied
    // (the MMA rows they feed are not stored)
    const int ct = threadIdx.x - 128;
    constexpr int NT = 32 * SG_NCONV;
    constexpr int AU = (SG_BM * 8 + NT - 1) / NT, BU = (BN * 8 + NT - 1) / NT;
    for (uint32_t g = 0;; ++g) {
      const int s = g % SG_STAGES;
      if (!sg_wait(&full[s], (g / SG_STAGES) & 1, abt)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      const SgMeta m = meta[s];
      if (!(m.flags & SG_STOP)) {
        unsigned char* st = smem + s * SG_STAGE_BYTES;
        float4 af[AU], bf[BU];
#pragma unroll
        for (int u = 0; u < AU; ++u) {
          const int i = ct + NT * u, r = i >> 3, c = i & 7;
          if (r < a.bmx) {
            const double2 v0 = *reinterpret_cast<const double2*>(st + r * (SG_BK * 8) + c * 32);
            const double2 v1 = *reinterpret_cast<const double2*>(st + r * (SG_BK * 8) + c * 32 + 16);
            af[u] = make_float4(sg_cvt(v0.x), sg_cvt(v0.y), sg_cvt(v1.x), sg_cvt(v1.y));
          }
        }
        const double* yt = reinterpret_cast<const double*>(st + SG_A_BYTES);
        const float cf = sg_cvt(m.cf);
        const int kq = a.q - m.kc * SG_BK;   // rows of Y at or past kq lie beyond this block
#pragma unroll
        for (int u = 0; u < BU; ++u) {
          const int i = ct + NT * u, j = i % BN, c = i / BN;
          if (c < 8) {
            const int k = 4 * c;
            bf[u] = make_float4(k < kq ? cf * sg_cvt(yt[k * BN + j]) : 0.0f,
                                k + 1 < kq ? cf * sg_cvt(yt[(k + 1) * BN + j]) : 0.0f,
                                k + 2 < kq ? cf * sg_cvt(yt[(k + 2) * BN + j]) : 0.0f,
                                k + 3 < kq ? cf * sg_cvt(yt[(k + 3) * BN + j]) : 0.0f);
          }
        }
        // every read of the FP64 tiles is done before their bytes are overwritten
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
#pragma unroll
        for (int u = 0; u < AU; ++u) {
          const int i = ct + NT * u, r = i >> 3, c = i & 7;
          if (r < a.bmx) {
            if constexpr (BF) {
              sg_store_bf16x3(st, st + SG_A_BYTES / 2, r, c, af[u]);
            } else {
              float4 hi, lo;
              sg_split(af[u].x, hi.x, lo.x);
              sg_split(af[u].y, hi.y, lo.y);
              sg_split(af[u].z, hi.z, lo.z);
              sg_split(af[u].w, hi.w, lo.w);
              const uint32_t off = sw128(r, c);
              *reinterpret_cast<float4*>(st + off) = hi;
              *reinterpret_cast<float4*>(st + SG_A_BYTES / 2 + off) = lo;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < BU; ++u) {
          const int i = ct + NT * u, j = i % BN, c = i / BN;
          if (c < 8) {
            if constexpr (BF) {
              sg_store_bf16x3(st + SG_A_BYTES, st + SG_A_BYTES + B_BYTES / 2, j, c, bf[u]);
            } else {
              float4 hi, lo;
              sg_split(bf[u].x, hi.x, lo.x);
              sg_split(bf[u].y, hi.y, lo.y);
              sg_split(bf[u].z, hi.z, lo.z);
              sg_split(bf[u].w, hi.w, lo.w);
              const uint32_t off = sw128(j, c);
              *reinterpret_cast<float4*>(st + SG_A_BYTES + off) = hi;
              *reinterpret_cast<float4*>(st + SG_A_BYTES + B_BYTES / 2 + off) = lo;
            }
          }
        }
        // generic-proxy writes made visible to the tensor cores' async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) sg_arrive(&conv[s]);
      if (m.flags & SG_STOP) break;
    }
  } else if (warp >= 4 + SG_NCONV) {
    // epilogue: warp 12 + q reads TMEM lanes / tile rows 32 q .. 32 q + 31 (the
    // lanes load the output offsets of 32 items at once); an item without
    // terms is a zero block and uses no accumulator
    const int qd = warp - (4 + SG_NCONV);
    const int G = gridDim.x;
    uint32_t n = 0;
    bool run = true;
    for (int base = blockIdx.x; base < nitems && run; base += 32 * G) {
      const int my = base + lane * G;
      int mnone = 1;
      long long mooff = 0;
      if (my < nitems) {
        const int seg = my / per_seg;
        mnone = a.seg_ptr[seg + 1] == a.seg_ptr[seg];
        mooff = a.out_by_seg ? (long long)seg * a.ors
                             : (long long)a.seg_or[seg] * a.ors + (long long)a.seg_oc[seg] * a.ocs;
      }
      for (int e = 0; e < 32; ++e) {
        const int it = base + e * G;
        if (it >= nitems) break;
        const int r = it % per_seg;
        const int i0 = (r / a.ntn) * SG_BM, j0 = (r % a.ntn) * BN;
        const bool none = __shfl_sync(0xffffffffu, mnone, e);
        const long long ooff = __shfl_sync(0xffffffffu, mooff, e);
        const int row = i0 + qd * 32 + lane;
        const bool rows_here = i0 + qd * 32 < a.p;   // this warp's quarter of the tile holds output rows
        if (none) {
          if (row < a.p && !a.accumulate) {
            double* o = a.O + ooff + (long long)row * a.os_i;
            for (int col = j0; col < min(a.s, j0 + BN); ++col) o[col] = 0.0;
          }
          continue;
        }
        const uint32_t buf = n % SG_NACC;
        int ok = 1;
        if (lane == 0) ok = sg_wait(&accf[buf], (n / SG_NACC) & 1, abt);
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          if (lane == 0) atomicExch(&abort_flag, 1);
          run = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (rows_here) {
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t rr[16];
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + buf * 128 + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                  "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                  "=r"(rr[14]), "=r"(rr[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < a.p) {
              double* o = a.O + ooff + (long long)row * a.os_i;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int col = j0 + c0 + jj;
                if (col < a.s) {
                  const double v = a.alpha * (double)__uint_as_float(rr[jj]);
                  o[col] = a.accumulate ? o[col] + v : v;
                }
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) sg_arrive(&acce[buf]);
        ++n;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) {
    atomicExch(a.err, 1);
    // the copies still in flight land before the shared memory is released
    for (int s = 0; s < SG_STAGES; ++s)
      if (issued[s]) mbar_wait(&full[s], (issued[s] - 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

bool make_map_f64(CUtensorMap* map, const double* base, long long rows, int cols, long long pitch, int box_cols,
                  int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 8};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool seg_mma_ok(const SegGemm& a) {
  if (!a.seg_ptr || a.splitk || a.tri || a.cs || a.kpart != 1) return false;
  if (a.xs_k != 1 || a.ys_j != 1 || a.os_j != 1) return false;
  if ((a.xc && a.xcs) || (a.yc && a.ycs)) return false;
  if (a.x_rows <= 0 || a.y_rows <= 0 || a.x_rows >= (1ll << 31) || a.y_rows >= (1ll << 31)) return false;
  if (a.xs_i % 2 || a.ys_k % 2 || a.q > a.xs_i || a.s > a.ys_k) return false;   // 16-byte row pitches
  if (a.xrs % a.xs_i || a.yrs % a.ys_k) return false;                          // blocks start on a row
  if ((uintptr_t)a.X % 16 || (uintptr_t)a.Y % 16) return false;
  // small blocks leave most of a 128-row MMA tile empty: the SIMT kernel is faster there
  if (a.p < 32 || a.q < 16 || a.s < 16) return false;
  return true;
}

bool seg_mma(const SegGemm& a, cudaStream_t st) {
  if (!seg_mma_ok(a)) return false;
  int* const err = tc_err_flag();
  if (!err) return false;
  const int bn = a.s <= 16 ? 16 : a.s <= 32 ? 32 : a.s <= 64 ? 64 : 128;
  CUtensorMap mX, mY;
  const int bmx = std::min(SG_BM, (a.p + 7) / 8 * 8);
  if (!make_map_f64(&mX, a.X, a.x_rows, a.q, a.xs_i, SG_BK, bmx) ||
      !make_map_f64(&mY, a.Y, a.y_rows, a.s, a.ys_k, bn, SG_BK))
    return false;
  SegMmaArgs g;
  g.seg_ptr = a.seg_ptr;
  g.seg_or = a.seg_or;
  g.seg_oc = a.seg_oc;
  g.xr = a.xr;
  g.yr = a.yr;
  g.cidx = a.cidx;
  g.coef = a.coef;
  g.xrow_unit = a.xrs / a.xs_i;
  g.yrow_unit = a.yrs / a.ys_k;
  g.p = a.p;
  g.q = a.q;
  g.s = a.s;
  g.nseg = a.nseg;
  g.ntm = (a.p + SG_BM - 1) / SG_BM;
  g.ntn = (a.s + bn - 1) / bn;
  g.out_by_seg = a.out_by_seg;
  g.accumulate = a.accumulate;
  g.bmx = bmx;
  g.ors = a.ors;
  g.ocs = a.ocs;
  g.os_i = a.os_i;
  g.O = a.O;
  g.alpha = a.alpha;
  g.err = err;
  static int nsm = [] {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  const long long items = (long long)g.nseg * g.ntm * g.ntn;
  if (items <= 0) return true;
  const int grid = int(std::min<long long>(items, nsm));
  auto go = [&](auto kern, int smem_bytes) {
    // the shared-memory limit is raised once per kernel variant (the first call
    // of each variant in the process; cudaFuncSetAttribute is thread-safe)
    static std::mutex attr_mu;
    static std::vector<const void*> raised;
    {
      std::lock_guard<std::mutex> lk(attr_mu);
      if (std::find(raised.begin(), raised.end(), (const void*)kern) == raised.end()) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        raised.push_back((const void*)kern);
      }
    }
    kern<<<grid, SG_THREADS, smem_bytes, st>>>(mX, mY, g);
  };
  if (g_tc_bf16) {
    if (bn == 16) go(seg_mma_3xtf32_kernel<16, true>, SgRing<16>::kSmem);
    else if (bn == 32) go(seg_mma_3xtf32_kernel<32, true>, SgRing<32>::kSmem);
    else if (bn == 64) go(seg_mma_3xtf32_kernel<64, true>, SgRing<64>::kSmem);
    else go(seg_mma_3xtf32_kernel<128, true>, SgRing<128>::kSmem);
  } else {
    if (bn == 16) go(seg_mma_3xtf32_kernel<16, false>, SgRing<16>::kSmem);
    else if (bn == 32) go(seg_mma_3xtf32_kernel<32, false>, SgRing<32>::kSmem);
    else if (bn == 64) go(seg_mma_3xtf32_kernel<64, false>, SgRing<64>::kSmem);
    else go(seg_mma_3xtf32_kernel<128, false>, SgRing<128>::kSmem);
  }
  ++g_count.launches;
  return true;
}

// 1 if any tensor-core GEMM timed out since the last call (then cleared)
int tc_gemm_take_error(cudaStream_t st) {
  int* e = tc_err_flag();
  if (!e) return 0;
  int v = 0;
  cudaMemcpyAsync(&v, e, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (v) cudaMemsetAsync(e, 0, sizeof(int), st);
  return v;
}

}  // namespace sgtn
