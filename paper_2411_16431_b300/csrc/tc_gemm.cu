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

#include <cstdint>
#include <mutex>

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
