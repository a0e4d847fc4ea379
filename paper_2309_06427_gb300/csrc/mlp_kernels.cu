// Kernels of the learned warm start (not in the paper): knot features, bf16
// tensor-core products with FP32 accumulation, the S^2-norm loss and its
// gradient, and Adam (Kingma & Ba, Algorithm 1).
#include <algorithm>

#include "mlp.h"

namespace sspcg {
namespace mlp {
namespace {

// ---------------------------------------------------------------------------
// Knot features.  A warp first stages its knot's data in shared memory with
// coalesced, independent loads (A_{k-1}, B_{k-1}, D_k^-1 compact, the
// diagonals and gamma_k), then writes the padded row from there.  Column
// pairs (c, c+1), c even, never straddle a segment or a padded matrix row
// (all segment starts and the row lengths 28 and 14 are even).
// ---------------------------------------------------------------------------
constexpr int kStA = 0, kStB = 784, kStPD = 1176, kStQp = 1960, kStRp = 1988, kStQ = 2002, kStG = 2030;
constexpr int kStDj = 2058, kStNx = 2086, kStZero = 2087;  // D_k^-1 gamma_k, nx / 28, a zero
constexpr int kStFloats = 2088;  // per warp (8,352 bytes)
constexpr int kFeatWarps = 4;

// dst[i] = src[i] for i < n <= MAXN: all loads issued before the stores.
template <int MAXN>
__device__ __forceinline__ void warp_copy(float *dst, const float *src, int n, int lane) {
  constexpr int T = (MAXN + 31) / 32;
  float v[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int i = lane + 32 * t;
    v[t] = i < n ? src[i] : 0.f;
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int i = lane + 32 * t;
    if (i < n) dst[i] = v[t];
  }
}

__device__ __forceinline__ void stage_knot(float *s, const ProbDesc &d, int k, const QpData &q, int lane) {
  const int m = d.nx, u = d.nu;
  if (k > 0) {
    warp_copy<kPadX * kPadX>(s + kStA, q.A + d.oA + (int64_t)(k - 1) * m * m, m * m, lane);
    if (u > 0) {
      warp_copy<kPadX * kPadU>(s + kStB, q.B + d.oB + (int64_t)(k - 1) * m * u, m * u, lane);
      if (lane < u) s[kStRp + lane] = q.rd[d.orr + (int64_t)(k - 1) * u + lane];
    }
    if (lane < m) s[kStQp + lane] = q.qd[d.oq + (int64_t)(k - 1) * m + lane];
  }
  warp_copy<kPadX * kPadX>(s + kStPD, q.PD + d.odiag + (int64_t)k * m * m, m * m, lane);
  if (lane < m) {
    s[kStQ + lane] = q.qd[d.oq + (int64_t)k * m + lane];
    s[kStG + lane] = q.gamma[d.ovec + (int64_t)k * m + lane];
  }
  __syncwarp();
}

__device__ __forceinline__ float2 feature_pair(int c, int m, int u, int k, const float *s, float dj0, float dj1) {
  float2 v = make_float2(0.f, 0.f);
  if (c < kOffB) {
    const int i = c / kPadX, j = c % kPadX;
    if (k > 0 && i < m) {
      if (j < m) v.x = s[kStA + i * m + j];
      if (j + 1 < m) v.y = s[kStA + i * m + j + 1];
    }
  } else if (c < kOffQp) {
    const int cc = c - kOffB, i = cc / kPadU, j = cc % kPadU;
    if (k > 0 && i < m) {
      if (j < u) v.x = s[kStB + i * u + j];
      if (j + 1 < u) v.y = s[kStB + i * u + j + 1];
    }
  } else if (c < kOffRp) {
    const int i = c - kOffQp;
    if (k > 0) {
      if (i < m) v.x = s[kStQp + i];
      if (i + 1 < m) v.y = s[kStQp + i + 1];
    }
  } else if (c < kOffQ) {
    const int i = c - kOffRp;
    if (k > 0) {
      if (i < u) v.x = s[kStRp + i];
      if (i + 1 < u) v.y = s[kStRp + i + 1];
    }
  } else if (c < kOffG) {
    const int i = c - kOffQ;
    if (i < m) v.x = s[kStQ + i];
    if (i + 1 < m) v.y = s[kStQ + i + 1];
  } else if (c < kOffDj) {
    const int i = c - kOffG;
    if (i < m) v.x = s[kStG + i];
    if (i + 1 < m) v.y = s[kStG + i + 1];
  } else if (c < kOffNx) {
    v.x = dj0;
    v.y = dj1;
  } else if (c == kOffNx) {
    v.x = (float)m / (float)kPadX;
  }
  return v;
}

// D_k^-1 gamma_k, component ``lane`` (zero for lane >= nx), from the staged PD block and gamma.
__device__ __forceinline__ float block_solve(const float *s, int m, int lane) {
  float acc = 0.f;
  if (lane < m) {
    const float *P = s + kStPD + lane * m;
    for (int j = 0; j < m; ++j) acc = fmaf(P[j], s[kStG + j], acc);
  }
  return acc;
}

constexpr int kPairIters = kIn / 64;  // 21 column pairs per lane

}  // namespace

// Gather table of the feature columns: for every (nx, nu) with nu <= 14, the stage index each column
// reads (kStZero for padding), in the column layout of feature_pair.
void build_feature_table(int16_t *tab) {
  for (int m = 1; m <= kPadX; ++m)
    for (int u = 0; u <= kPadU; ++u) {
      int16_t *t = tab + ((int64_t)(m - 1) * (kPadU + 1) + u) * kIn;
      for (int c = 0; c < kIn; ++c) {
        int idx = kStZero;
        if (c < kOffB) {
          const int i = c / kPadX, j = c % kPadX;
          if (i < m && j < m) idx = kStA + i * m + j;
        } else if (c < kOffQp) {
          const int cc = c - kOffB, i = cc / kPadU, j = cc % kPadU;
          if (i < m && j < u) idx = kStB + i * u + j;
        } else if (c < kOffRp) {
          if (c - kOffQp < m) idx = kStQp + (c - kOffQp);
        } else if (c < kOffQ) {
          if (c - kOffRp < u) idx = kStRp + (c - kOffRp);
        } else if (c < kOffG) {
          if (c - kOffQ < m) idx = kStQ + (c - kOffQ);
        } else if (c < kOffDj) {
          if (c - kOffG < m) idx = kStG + (c - kOffG);
        } else if (c < kOffNx) {
          if (c - kOffDj < m) idx = kStDj + (c - kOffDj);
        } else if (c == kOffNx) {
          idx = kStNx;
        }
        t[c] = (int16_t)idx;
      }
    }
}

namespace {

// One warp per knot row: stage the knot's data (zeros for the k - 1 blocks of row 0), then lane l writes
// columns 64 i + 2 l, +1, each gathered from the stage through the table of the problem's (nx, nu).
__global__ void __launch_bounds__(kFeatWarps * 32) features_kernel(RowSpan rs, QpData q, const float *__restrict__ mu,
                                                                   const float *__restrict__ isd,
                                                                   const int16_t *__restrict__ tab,
                                                                   bf16 *__restrict__ X) {
  __shared__ __align__(16) float stage[kFeatWarps][kStFloats];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * kFeatWarps + wl;
  if (r >= rs.nrows) return;  // warp-uniform
  const int2 ref = rs.kref[rs.row0 + r];
  const ProbDesc d = rs.ps.get(ref.x);
  const int k = ref.y, m = d.nx, u = d.nu;
  float *s = stage[wl];
  if (k == 0) {  // no A_{k-1}, B_{k-1}, diag Q_{k-1}, diag R_{k-1}: their columns read zeros
    for (int e = lane; e < m * m; e += 32) s[kStA + e] = 0.f;
    for (int e = lane; e < m * u; e += 32) s[kStB + e] = 0.f;
    if (lane < m) s[kStQp + lane] = 0.f;
    if (lane < u) s[kStRp + lane] = 0.f;
  }
  stage_knot(s, d, k, q, lane);  // ends with __syncwarp
  const float dj = block_solve(s, m, lane);  // zero for lane >= nx
  if (lane < kPadX) s[kStDj + lane] = dj;
  if (lane == 0) {
    s[kStNx] = (float)m / (float)kPadX;
    s[kStZero] = 0.f;
  }
  __syncwarp();
  const int16_t *t = tab + ((int64_t)(m - 1) * (kPadU + 1) + u) * kIn;
  __nv_bfloat162 *out = reinterpret_cast<__nv_bfloat162 *>(X + r * kIn);
#pragma unroll
  for (int it = 0; it < kPairIters; ++it) {
    const int c = it * 64 + 2 * lane;
    const short2 id = *reinterpret_cast<const short2 *>(t + c);
    const float2 mm = *reinterpret_cast<const float2 *>(mu + c);
    const float2 is = *reinterpret_cast<const float2 *>(isd + c);
    const float vx = (s[id.x] - mm.x) * is.x;
    const float vy = (s[id.y] - mm.y) * is.y;
    out[c >> 1] = __floats2bfloat162_rn(vx, vy);
  }
}

// Per-warp FP64 column sums and sums of squares of the raw features.
__global__ void __launch_bounds__(kFeatWarps * 32) feature_stats_kernel(RowSpan rs, QpData q,
                                                                        double *__restrict__ part) {
  __shared__ __align__(16) float stage[kFeatWarps][kStFloats];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * kFeatWarps + wl;
  const int64_t nw = (int64_t)gridDim.x * kFeatWarps;
  float *s = stage[wl];
  double sm[kPairIters][2], ss[kPairIters][2];
#pragma unroll
  for (int it = 0; it < kPairIters; ++it) sm[it][0] = sm[it][1] = ss[it][0] = ss[it][1] = 0.0;
  for (int64_t r = w; r < rs.nrows; r += nw) {
    const int2 ref = rs.kref[rs.row0 + r];
    const ProbDesc d = rs.ps.get(ref.x);
    const int k = ref.y, m = d.nx, u = d.nu;
    __syncwarp();  // the previous row's reads of the stage are done
    stage_knot(s, d, k, q, lane);
    const float dj = block_solve(s, m, lane);
#pragma unroll
    for (int it = 0; it < kPairIters; ++it) {
      const int c = it * 64 + 2 * lane;
      float dj0 = 0.f, dj1 = 0.f;
      if (it >= kOffDj / 64) {
        const int sidx = min(max(c - kOffDj, 0), 30);
        dj0 = __shfl_sync(0xffffffffu, dj, sidx);
        dj1 = __shfl_sync(0xffffffffu, dj, sidx + 1);
      }
      const float2 v = feature_pair(c, m, u, k, s, dj0, dj1);
      sm[it][0] += v.x; sm[it][1] += v.y;
      ss[it][0] += (double)v.x * v.x; ss[it][1] += (double)v.y * v.y;
    }
  }
  double *o = part + w * 2 * kIn;
#pragma unroll
  for (int it = 0; it < kPairIters; ++it) {
    const int c = it * 64 + 2 * lane;
    o[c] = sm[it][0]; o[c + 1] = sm[it][1];
    o[kIn + c] = ss[it][0]; o[kIn + c + 1] = ss[it][1];
  }
}

// mu and 1/sigma per column; a column whose sigma is at most 1e-6 of its RMS is constant (1/sigma = 0).
__global__ void stats_finish_kernel(const double *__restrict__ part, int warps, int64_t rows, float *mu,
                                    float *isd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kIn) return;
  double s = 0.0, ss = 0.0;
  for (int w = 0; w < warps; ++w) {
    s += part[(int64_t)w * 2 * kIn + c];
    ss += part[(int64_t)w * 2 * kIn + kIn + c];
  }
  const double n = rows > 0 ? (double)rows : 1.0;
  const double m = s / n, ms = ss / n;
  const double var = fmax(ms - m * m, 0.0);
  const double sig = sqrt(var);
  mu[c] = (float)m;
  isd[c] = sig <= 1e-6 * sqrt(ms) ? 0.f : (float)(1.0 / sig);
}

// ---------------------------------------------------------------------------
// bf16 tensor-core products: mma.sync m16n8k16, operands staged by cp.async
// (16-byte chunks, zero fill past the last row), fragments by ldmatrix.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kBK = 32;        // contraction step
constexpr int kLdNT = kBK + 8;  // padded smem row (bf16): 80 bytes, conflict-free ldmatrix

// C[M][N] = epi(A[M][K] B[N][K]^T); N % BN == 0, K % 32 == 0.
template <int BM, int BN, int WM, int WN, int EPI>
__global__ void __launch_bounds__(WM *WN * 32) gemm_nt_kernel(const bf16 *__restrict__ A, const bf16 *__restrict__ B,
                                                              int64_t M, int N, int K, const float *__restrict__ bias,
                                                              const bf16 *__restrict__ mask, bf16 *__restrict__ Cb,
                                                              float *__restrict__ Cf) {
  constexpr int T = WM * WN * 32, TM = BM / WM, TN = BN / WN, MT = TM / 16, NT = TN / 8;
  static_assert(NT % 2 == 0, "two n8 tiles per ldmatrix");
  __shared__ __align__(128) bf16 As[2][BM][kLdNT];
  __shared__ __align__(128) bf16 Bs[2][BN][kLdNT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WM, wn = warp / WM;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int KT = K / kBK;

  auto load = [&](int stage, int k0) {
    for (int i = tid; i < BM * 4; i += T) {
      const int r = i >> 2, ch = i & 3;
      const int64_t gr = m0 + r;
      const bf16 *src = A + (gr < M ? gr : M - 1) * (int64_t)K + k0 + ch * 8;
      cp_async16(&As[stage][r][ch * 8], src, gr < M ? 16 : 0);
    }
    for (int i = tid; i < BN * 4; i += T) {
      const int r = i >> 2, ch = i & 3;
      cp_async16(&Bs[stage][r][ch * 8], B + (int64_t)(n0 + r) * K + k0 + ch * 8, 16);
    }
  };

  float acc[MT][NT][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  load(0, 0);
  cp_async_commit();
  for (int kt = 0; kt < KT; ++kt) {
    if (kt + 1 < KT) {
      load((kt + 1) & 1, (kt + 1) * kBK);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int s = kt & 1;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t af[MT][4];
#pragma unroll
      for (int a = 0; a < MT; ++a) {
        const int j = lane >> 3;
        const int row = wm * TM + a * 16 + (lane & 7) + (j & 1) * 8;
        ldsm_x4(af[a], &As[s][row][kk + (j >> 1) * 8]);
      }
#pragma unroll
      for (int b = 0; b < NT; b += 2) {
        const int j = lane >> 3;
        const int row = wn * TN + b * 8 + (lane & 7) + (j >> 1) * 8;
        uint32_t bf[4];
        ldsm_x4(bf, &Bs[s][row][kk + (j & 1) * 8]);
#pragma unroll
        for (int a = 0; a < MT; ++a) {
          mma_bf16(acc[a][b], af[a], bf[0], bf[1]);
          mma_bf16(acc[a][b + 1], af[a], bf[2], bf[3]);
        }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      const int col = n0 + wn * TN + b * 8 + 2 * (lane & 3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = m0 + wm * TM + a * 16 + (lane >> 2) + h * 8;
        if (row >= M) continue;
        float v0 = acc[a][b][2 * h], v1 = acc[a][b][2 * h + 1];
        const int64_t o = row * N + col;
        if (EPI == kEpiBiasRelu) {
          v0 = fmaxf(v0 + bias[col], 0.f);
          v1 = fmaxf(v1 + bias[col + 1], 0.f);
          *reinterpret_cast<__nv_bfloat162 *>(Cb + o) = __floats2bfloat162_rn(v0, v1);
        } else if (EPI == kEpiBiasF32) {
          *reinterpret_cast<float2 *>(Cf + o) = make_float2(v0 + bias[col], v1 + bias[col + 1]);
        } else {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + o);
          v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
          v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
          *reinterpret_cast<__nv_bfloat162 *>(Cb + o) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
}

// part[s][N1][N2] = sum over the rows m of split s of G[m][n1] X[m][n2]; 4 warps as 2 x 2.
template <int BM, int BN>
__global__ void __launch_bounds__(128) gemm_tn_kernel(const bf16 *__restrict__ G, int N1, const bf16 *__restrict__ X,
                                                      int N2, int64_t M, int64_t rps, float *__restrict__ part) {
  constexpr int TM = BM / 2, TN = BN / 2, MT = TM / 16, NT = TN / 8;
  constexpr int LA = BM + 8, LB = BN + 8;
  __shared__ __align__(128) bf16 Gs[2][kBK][LA];
  __shared__ __align__(128) bf16 Xs[2][kBK][LB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int n2_0 = blockIdx.x * BN, n1_0 = blockIdx.y * BM;
  const int64_t r_begin = (int64_t)blockIdx.z * rps;
  const int64_t r_end = r_begin + rps < M ? r_begin + rps : M;
  const int KT = (int)((r_end - r_begin + kBK - 1) / kBK);

  auto load = [&](int stage, int64_t r0) {
    for (int i = tid; i < kBK * (BM / 8); i += 128) {
      const int r = i / (BM / 8), ch = i % (BM / 8);
      const int64_t gr = r0 + r;
      const bool ok = gr < r_end;
      cp_async16(&Gs[stage][r][ch * 8], G + (ok ? gr : r_begin) * N1 + n1_0 + ch * 8, ok ? 16 : 0);
    }
    for (int i = tid; i < kBK * (BN / 8); i += 128) {
      const int r = i / (BN / 8), ch = i % (BN / 8);
      const int64_t gr = r0 + r;
      const bool ok = gr < r_end;
      cp_async16(&Xs[stage][r][ch * 8], X + (ok ? gr : r_begin) * N2 + n2_0 + ch * 8, ok ? 16 : 0);
    }
  };

  float acc[MT][NT][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  if (KT > 0) {
    load(0, r_begin);
    cp_async_commit();
  }
  for (int kt = 0; kt < KT; ++kt) {
    if (kt + 1 < KT) {
      load((kt + 1) & 1, r_begin + (int64_t)(kt + 1) * kBK);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int s = kt & 1;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      const int j = lane >> 3;
      uint32_t af[MT][4];
#pragma unroll
      for (int a = 0; a < MT; ++a)
        ldsm_x4_t(af[a], &Gs[s][kk + (lane & 7) + (j >> 1) * 8][wm * TM + a * 16 + (j & 1) * 8]);
#pragma unroll
      for (int b = 0; b < NT; b += 2) {
        uint32_t bf[4];
        ldsm_x4_t(bf, &Xs[s][kk + (lane & 7) + (j & 1) * 8][wn * TN + b * 8 + (j >> 1) * 8]);
#pragma unroll
        for (int a = 0; a < MT; ++a) {
          mma_bf16(acc[a][b], af[a], bf[0], bf[1]);
          mma_bf16(acc[a][b + 1], af[a], bf[2], bf[3]);
        }
      }
    }
    __syncthreads();
  }

  float *out = part + (int64_t)blockIdx.z * N1 * N2;
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      const int col = n2_0 + wn * TN + b * 8 + 2 * (lane & 3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = n1_0 + wm * TM + a * 16 + (lane >> 2) + h * 8;
        *reinterpret_cast<float2 *>(out + (int64_t)row * N2 + col) = make_float2(acc[a][b][2 * h], acc[a][b][2 * h + 1]);
      }
    }
}

__global__ void colsum_kernel(const bf16 *__restrict__ Y, int64_t M, int N, int64_t rps, float *__restrict__ part) {
  const int c = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * rps;
  const int64_t r1 = r0 + rps < M ? r0 + rps : M;
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += __bfloat162float(Y[r * N + c]);
  part[(int64_t)blockIdx.x * N + c] = s;
}

__global__ void reduce_splits_kernel(const float *__restrict__ part, int64_t splits, int64_t n, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int64_t k = 0; k < splits; ++k) s += part[k * n + i];
  out[i] = s;
}

// ---------------------------------------------------------------------------
// Loss: one CTA per problem.  u = S (lambda0 - lambda*), with S's blocks D, E
// (S_{k,k-1} = E_{k-1} in the packed [N][nx][nx] layout, S_{k,k+1} = its
// transpose); then dL/dlambda0 = 2 S u / (P ||gamma||^2).
// ---------------------------------------------------------------------------
constexpr int kLossThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double *slots) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) slots[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += slots[i];
  return s;
}

// y_e for e = k nx + i of the block tridiagonal product with x given by xk(kk, j).
template <typename XF>
__device__ __forceinline__ float bt_row(const ProbDesc &d, const float *D, const float *E, int k, int i, XF xk) {
  const int m = d.nx;
  const float *Dr = D + d.odiag + (int64_t)k * m * m + (int64_t)i * m;
  float s = 0.f;
  for (int j = 0; j < m; ++j) s = fmaf(Dr[j], xk(k, j), s);
  if (k > 0) {
    const float *Er = E + d.ooff + (int64_t)(k - 1) * m * m + (int64_t)i * m;
    for (int j = 0; j < m; ++j) s = fmaf(Er[j], xk(k - 1, j), s);
  }
  if (k < d.N) {
    const float *Ec = E + d.ooff + (int64_t)k * m * m + i;
    for (int j = 0; j < m; ++j) s = fmaf(Ec[(int64_t)j * m], xk(k + 1, j), s);
  }
  return s;
}

__global__ void __launch_bounds__(kLossThreads) loss_u_kernel(LossArgs a) {
  __shared__ double slots[kLossThreads / 32];
  const int p = a.p0 + blockIdx.x;
  const ProbDesc d = a.ps.get(p);
  const int m = d.nx;
  const int64_t rows0 = a.knot_start[p] - a.row0;
  const int64_t ne = (int64_t)(d.N + 1) * m;
  auto err = [&](int k, int j) {
    return a.Y[(rows0 + k) * kOut + j] - a.lamstar[d.ovec + (int64_t)k * m + j];
  };
  double uu = 0.0, gg = 0.0;
  for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
    const int k = (int)(e / m), i = (int)(e % m);
    const float u = bt_row(d, a.D, a.E, k, i, err);
    a.U[(rows0 + k) * kOut + i] = u;
    uu += (double)u * u;
    const float g = a.gamma[d.ovec + e];
    gg += (double)g * g;
  }
  uu = block_sum_d(uu, slots);
  gg = block_sum_d(gg, slots);
  if (threadIdx.x == 0) {
    a.uu[blockIdx.x] = uu;
    a.gg[blockIdx.x] = gg > 0.0 ? gg : 1.0;
  }
}

__global__ void __launch_bounds__(kLossThreads) loss_grad_kernel(LossArgs a) {
  const int p = a.p0 + blockIdx.x;
  const ProbDesc d = a.ps.get(p);
  const int m = d.nx;
  const int64_t rows0 = a.knot_start[p] - a.row0;
  const float scale = (float)(2.0 / ((double)(a.p1 - a.p0) * a.gg[blockIdx.x]));
  auto uk = [&](int k, int j) { return a.U[(rows0 + k) * kOut + j]; };
  const int64_t ne = (int64_t)(d.N + 1) * kOut;
  for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
    const int k = (int)(e / kOut), i = (int)(e % kOut);
    float g = 0.f;
    if (i < m) g = scale * bt_row(d, a.D, a.E, k, i, uk);
    a.dY[(rows0 + k) * kOut + i] = __float2bfloat16_rn(g);
  }
}

__global__ void loss_total_kernel(const double *uu, const double *gg, int P, double *loss) {
  __shared__ double slots[32];
  double s = 0.0;
  // fixed summation order: thread t takes problems t, t + blockDim, ...
  for (int i = threadIdx.x; i < P; i += blockDim.x) s += uu[i] / gg[i];
  s = block_sum_d(s, slots);
  if (threadIdx.x == 0) *loss = s / (P > 0 ? P : 1);
}

// ---------------------------------------------------------------------------
// Adam on FP32 master weights, then the bf16 copies the products read:
// W1, W2, W3 as stored and W2^T [256][256], W3^T [256][32] for the backward
// products.
// ---------------------------------------------------------------------------
__global__ void adam_kernel(AdamArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  float w = a.w[i];
  if (a.update) {
    const float g = a.g[i];
    const float m = a.beta1 * a.m[i] + (1.f - a.beta1) * g;
    const float v = a.beta2 * a.v[i] + (1.f - a.beta2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    const float mh = m / a.bc1, vh = v / a.bc2;
    w -= a.lr * mh / (sqrtf(vh) + a.eps);
    a.w[i] = w;
  }
  const bf16 wb = __float2bfloat16_rn(w);
  if (i < kB1) {
    a.W1b[i - kW1] = wb;
  } else if (i >= kW2 && i < kB2) {
    const int64_t j = i - kW2, o = j / kHid, c = j % kHid;
    a.W2b[j] = wb;
    a.W2t[c * kHid + o] = wb;
  } else if (i >= kW3 && i < kB3) {
    const int64_t j = i - kW3, o = j / kHid, c = j % kHid;
    a.W3b[j] = wb;
    a.W3t[c * kOut + o] = wb;
  }
}

__global__ void scatter_lambda_kernel(RowSpan rs, const float *__restrict__ Y, float *__restrict__ lambda) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rs.nrows * kOut) return;
  const int64_t r = e / kOut;
  const int i = (int)(e % kOut);
  const int2 ref = rs.kref[rs.row0 + r];
  const ProbDesc d = rs.ps.get(ref.x);
  if (i < d.nx) lambda[d.ovec + (int64_t)ref.y * d.nx + i] = Y[r * kOut + i];
}

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t launch_features(const RowSpan &rs, const QpData &q, const float *mu, const float *isd,
                            const int16_t *tab, bf16 *X, cudaStream_t st) {
  if (rs.nrows <= 0) return cudaSuccess;
  features_kernel<<<(unsigned)cdiv64(rs.nrows, kFeatWarps), kFeatWarps * 32, 0, st>>>(rs, q, mu, isd, tab, X);
  return cudaGetLastError();
}

int feature_stats_warps(int sms) { return sms * 8 * 2; }

cudaError_t launch_feature_stats(const RowSpan &rs, const QpData &q, double *part, int warps, cudaStream_t st) {
  feature_stats_kernel<<<warps / kFeatWarps, kFeatWarps * 32, 0, st>>>(rs, q, part);
  return cudaGetLastError();
}

cudaError_t launch_stats_finish(const double *part, int warps, int64_t rows, float *mu, float *isd,
                                cudaStream_t st) {
  stats_finish_kernel<<<(kIn + 127) / 128, 128, 0, st>>>(part, warps, rows, mu, isd);
  return cudaGetLastError();
}

template <int BM, int BN, int WM, int WN>
static cudaError_t gemm_nt_tiles(int epi, const bf16 *A, const bf16 *B, int64_t M, int N, int K, const float *bias,
                                 const bf16 *mask, bf16 *Cb, float *Cf, cudaStream_t st) {
  const dim3 grid((unsigned)(N / BN), (unsigned)cdiv64(M, BM));
  if (epi == kEpiBiasRelu)
    gemm_nt_kernel<BM, BN, WM, WN, kEpiBiasRelu><<<grid, WM * WN * 32, 0, st>>>(A, B, M, N, K, bias, mask, Cb, Cf);
  else if (epi == kEpiBiasF32)
    gemm_nt_kernel<BM, BN, WM, WN, kEpiBiasF32><<<grid, WM * WN * 32, 0, st>>>(A, B, M, N, K, bias, mask, Cb, Cf);
  else
    gemm_nt_kernel<BM, BN, WM, WN, kEpiMask><<<grid, WM * WN * 32, 0, st>>>(A, B, M, N, K, bias, mask, Cb, Cf);
  return cudaGetLastError();
}

cudaError_t launch_gemm_nt(int epi, const bf16 *A, const bf16 *B, int64_t M, int N, int K, const float *bias,
                           const bf16 *mask, bf16 *Cb, float *Cf, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  if (K % kBK != 0) return cudaErrorInvalidValue;
  if (N % 128 == 0) return gemm_nt_tiles<128, 128, 4, 2>(epi, A, B, M, N, K, bias, mask, Cb, Cf, st);
  if (N % 32 == 0) return gemm_nt_tiles<128, 32, 8, 1>(epi, A, B, M, N, K, bias, mask, Cb, Cf, st);
  return cudaErrorInvalidValue;
}

int64_t gemm_tn_splits(int64_t M) { return M > 0 ? std::min<int64_t>(cdiv64(M, kRowsPerSplit), kMaxSplits) : 0; }

// Rows per split: a multiple of the contraction step, at least kRowsPerSplit.
static int64_t rows_per_split(int64_t M) {
  const int64_t splits = gemm_tn_splits(M);
  return ((cdiv64(M, splits) + kBK - 1) / kBK) * kBK;
}

cudaError_t launch_gemm_tn(const bf16 *G, int N1, const bf16 *X, int N2, int64_t M, float *part, cudaStream_t st) {
  const int64_t splits = gemm_tn_splits(M);
  if (splits == 0) return cudaSuccess;
  if (N2 % 64 != 0) return cudaErrorInvalidValue;
  const int64_t rps = rows_per_split(M);
  if (N1 % 64 == 0) {
    gemm_tn_kernel<64, 64><<<dim3(N2 / 64, N1 / 64, (unsigned)splits), 128, 0, st>>>(G, N1, X, N2, M, rps, part);
  } else if (N1 % 32 == 0) {
    gemm_tn_kernel<32, 64><<<dim3(N2 / 64, N1 / 32, (unsigned)splits), 128, 0, st>>>(G, N1, X, N2, M, rps, part);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_colsum(const bf16 *Y, int64_t M, int N, float *part, cudaStream_t st) {
  const int64_t chunks = gemm_tn_splits(M);
  if (chunks == 0) return cudaSuccess;
  colsum_kernel<<<(unsigned)chunks, N, 0, st>>>(Y, M, N, rows_per_split(M), part);
  return cudaGetLastError();
}

cudaError_t launch_reduce_splits(const float *part, int64_t splits, int64_t n, float *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (splits == 0) return cudaMemsetAsync(out, 0, sizeof(float) * n, st);
  reduce_splits_kernel<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(part, splits, n, out);
  return cudaGetLastError();
}

cudaError_t launch_loss(const LossArgs &a, cudaStream_t st) {
  const int P = a.p1 - a.p0;
  if (P <= 0) return cudaSuccess;
  loss_u_kernel<<<P, kLossThreads, 0, st>>>(a);
  loss_grad_kernel<<<P, kLossThreads, 0, st>>>(a);
  loss_total_kernel<<<1, 256, 0, st>>>(a.uu, a.gg, P, a.loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st) {
  adam_kernel<<<(unsigned)cdiv64(kParams, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter_lambda(const RowSpan &rs, const float *Y, float *lambda, cudaStream_t st) {
  if (rs.nrows <= 0) return cudaSuccess;
  scatter_lambda_kernel<<<(unsigned)cdiv64(rs.nrows * kOut, 256), 256, 0, st>>>(rs, Y, lambda);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace sspcg
