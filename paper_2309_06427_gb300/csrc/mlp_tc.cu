// Warm-start network products on the 5th-generation tensor cores:
// C[M][N] = epilogue(A[M][K] B[N][K]^T), bf16 operands, FP32 accumulation in
// tensor memory.  One CTA (4 warps) per 128-row tile and the whole N (256 or
// 32): warp 0 streams A and B tiles of 64 columns (128 bytes) into a ring of
// shared-memory stages with TMA (128-byte swizzle); warp 1 issues
// tcgen05.mma (M = 128, K = 16 per instruction) from one thread and
// releases each stage with tcgen05.commit; then all four warps read the
// accumulators (tcgen05.ld, one TMEM lane per row) and apply the epilogue.
// Every mbarrier wait is bounded: on expiry the kernel records an error code,
// skips its remaining work, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "mlp.h"

namespace sspcg {
namespace mlp {
namespace {

constexpr int kTcM = 128;          // rows per tile (TMEM lanes)
constexpr int kTcK = 64;           // columns per stage: one 128-byte swizzle row of bf16
constexpr int kTcThreads = 128;
constexpr uint32_t kSpinLimit = 1u << 26;  // polls of one mbarrier wait (well over a second)

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// Wait until the phase of parity ``parity`` has completed; false when the bound expires.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = su32(bar);
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
  const uint64_t addr = su32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 accumulator, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4)                       // accumulator format F32
         | (1u << 7)                     // A format BF16
         | (1u << 10)                    // B format BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int N>
struct TcCfg {
  static constexpr int kStages = N >= 256 ? 4 : 6;
  static constexpr int kABytes = kTcM * kTcK * 2;  // 16 KB
  static constexpr int kBBytes = N * kTcK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kTmemCols = N < 32 ? 32 : N;  // power of two >= 32
  static constexpr int kSmem = kStages * kStageBytes + 1024 /*alignment*/ + 256 /*barriers*/;
};

template <int N, int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
    gemm_nt_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t M,
                      int K, const float *__restrict__ bias, bf16 *__restrict__ Cb, float *__restrict__ Cf,
                      int *__restrict__ err) {
  using C = TcCfg<N>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *stage_base = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::kStages * C::kStageBytes);
  uint64_t *empty = full + C::kStages;
  uint64_t *acc_full = empty + C::kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_full + 1);
  __shared__ int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTcM;
  const int KT = K / kTcK;

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of A rows [m0, m0 + 128) and all N rows of B, 64 columns per stage
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % C::kStages;
      if (kt >= C::kStages && !mbar_wait(&empty[s], ((kt / C::kStages) - 1) & 1)) {
        atomicExch(&failed, 1);
        break;
      }
      uint8_t *a = stage_base + s * C::kStageBytes;
      uint8_t *b = a + C::kABytes;
      mbar_expect_tx(&full[s], C::kStageBytes);
      tma_load_2d(a, &mapA, kt * kTcK, (int)m0, &full[s]);
      tma_load_2d(b, &mapB, kt * kTcK, 0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc(kTcM, N);
    bool ok = true;
    for (int kt = 0; kt < KT && ok; ++kt) {
      const int s = kt % C::kStages;
      if (!mbar_wait(&full[s], (kt / C::kStages) & 1)) {
        atomicExch(&failed, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint8_t *a = stage_base + s * C::kStageBytes;
      const uint8_t *b = a + C::kABytes;
#pragma unroll
      for (int k = 0; k < kTcK / 16; ++k)
        mma_issue(tmem, smem_desc(a + k * 32), smem_desc(b + k * 32), idesc, (kt > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty[s]);  // stage free once these products have read it
    }
    mma_commit(acc_full);  // accumulators complete
  }
  __syncwarp();

  // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
  bool ready = mbar_wait(acc_full, 0);
  if (!ready) atomicExch(&failed, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (!failed) {
    const int row_in_tile = warp * 32 + lane;
    const int64_t row = m0 + row_in_tile;
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + (uint32_t)c0, v);
      if (row < M) {
        if (EPI == kEpiBiasRelu) {
          uint32_t packed[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float x0 = fmaxf(v[2 * i] + bias[c0 + 2 * i], 0.f);
            const float x1 = fmaxf(v[2 * i + 1] + bias[c0 + 2 * i + 1], 0.f);
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            packed[i] = *reinterpret_cast<const uint32_t *>(&h);
          }
          uint4 *dst = reinterpret_cast<uint4 *>(Cb + row * N + c0);
          dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        } else {
          float4 *dst = reinterpret_cast<float4 *>(Cf + row * N + c0);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            dst[i] = make_float4(v[4 * i] + bias[c0 + 4 * i], v[4 * i + 1] + bias[c0 + 4 * i + 1],
                                 v[4 * i + 2] + bias[c0 + 4 * i + 2], v[4 * i + 3] + bias[c0 + 4 * i + 3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::kTmemCols));
  }
  if (threadIdx.x == 0 && failed) atomicExch(err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D bf16 tensor [rows][cols] (row-major), box of kTcK columns x box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap *map, const bf16 *base, int64_t rows, int cols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(bf16)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N, int EPI>
cudaError_t launch_tc(const CUtensorMap &ma, const CUtensorMap &mb, int64_t M, int K, const float *bias, bf16 *Cb,
                      float *Cf, int *err, cudaStream_t st) {
  using C = TcCfg<N>;
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = smem_attr_once(attr_done, gemm_nt_tc_kernel<N, EPI>, C::kSmem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((M + kTcM - 1) / kTcM);
  gemm_nt_tc_kernel<N, EPI><<<grid, kTcThreads, C::kSmem, st>>>(ma, mb, M, K, bias, Cb, Cf, err);
  return cudaGetLastError();
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

cudaError_t launch_gemm_nt_tc(int epi, const bf16 *A, const bf16 *B, int64_t M, int N, int K, const float *bias,
                              bf16 *Cb, float *Cf, int *err, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  if (K % kTcK != 0 || K <= 0) return cudaErrorInvalidValue;
  if (!(N == 256 || N == 32)) return cudaErrorInvalidValue;
  if (!(epi == kEpiBiasRelu || epi == kEpiBiasF32)) return cudaErrorInvalidValue;
  // TMA needs 16-byte aligned bases and row strides (K * 2 bytes: K % 64 == 0)
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u)) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, kTcM) || !make_map(&mb, B, N, K, N)) return cudaErrorInvalidValue;
  if (N == 256)
    return epi == kEpiBiasRelu ? launch_tc<256, kEpiBiasRelu>(ma, mb, M, K, bias, Cb, Cf, err, st)
                               : launch_tc<256, kEpiBiasF32>(ma, mb, M, K, bias, Cb, Cf, err, st);
  return epi == kEpiBiasRelu ? launch_tc<32, kEpiBiasRelu>(ma, mb, M, K, bias, Cb, Cf, err, st)
                             : launch_tc<32, kEpiBiasF32>(ma, mb, M, K, bias, Cb, Cf, err, st);
}

}  // namespace mlp
}  // namespace sspcg
