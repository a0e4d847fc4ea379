// Fused PCG kernel: one CTA runs the whole preconditioned CG loop of one
// problem (Sec. II-B), with S p and Phi^-1 r as block-tridiagonal products
// and the dot products reduced by warp shuffles.  Included by the per-nx
// instantiation units.
//
// Thread mapping: thread t owns rows t, t + T, t + 2T, ... of the
// (N+1)*nx unknowns; row = k*nx + i is row i of block row k.
//
// Per iteration (textbook PCG, Saad Alg. 9.1):
//   w = S p                 (QP form: v = G^-1 C^T p, sync, w = C v)
//   alpha = (r.z) / (p.w)   block reduction
//   x += alpha p, r -= alpha w, sync
//   z = Phi^-1 r, (r.z), (r.r) block reduction
//   beta = (r.z)new / (r.z)old, p = z + beta p, sync
// Stop before an iteration once r.r <= tol^2 gamma.gamma.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace sspcg {

template <bool RES>
__device__ __forceinline__ float ldm(const float *p) {
  if constexpr (RES) return *p;
  else return __ldg(p);
}

// Accumulators of the three reduction modes.
template <int RED> struct Red;
template <> struct Red<kRedF32> {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.0f; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return fmaf(a, b, acc); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float tof(T v) { return v; }
  static __device__ __forceinline__ double tod(T v) { return (double)v; }
};
template <> struct Red<kRedDf> {
  using T = df;
  static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return df_fma(acc, a, b); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float tof(T v) { return __fadd_rn(v.hi, v.lo); }
  static __device__ __forceinline__ double tod(T v) { return df_to_double(v); }
};
template <> struct Red<kRedF64> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return ::fma((double)a, (double)b, acc); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float tof(T v) { return (float)v; }
  static __device__ __forceinline__ double tod(T v) { return v; }
};

// Block-wide sum of K accumulators: warp butterflies, one slot per warp,
// one barrier, then every warp sums the slots in the same order, so all
// threads hold bit-identical results.
template <int RED, int K>
__device__ __forceinline__ void block_sum(typename Red<RED>::T (&v)[K], typename Red<RED>::T *slots) {
  using R = Red<RED>;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int e = 0; e < K; ++e) v[e] = R::sum(v[e]);
  if (lane == 0) {
#pragma unroll
    for (int e = 0; e < K; ++e) slots[e * 32 + wid] = v[e];
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < K; ++e) v[e] = R::sum(lane < nw ? slots[e * 32 + lane] : R::zero());
}

// Row (k, i) of a block-tridiagonal symmetric matrix times v:
//   Md: diagonal blocks (symmetric; read by column so that consecutive i are
//   consecutive addresses), Mo: sub-diagonal blocks, Mo[k-1] = M(k, k-1),
//   M(k, k+1) = Mo[k]^T.  ld: row stride of the blocks.
template <int NX, bool RES>
__device__ __forceinline__ float bt_row(const float *Md, const float *Mo, int ld, int N, int k, int i,
                                        const float *v) {
  const float *vk = v + k * NX;
  const float *dk = Md + (int64_t)k * NX * ld + i;
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < NX; ++j) acc = fmaf(ldm<RES>(dk + j * ld), vk[j], acc);
  if (k > 0) {
    const float *ok = Mo + (int64_t)(k - 1) * NX * ld + i * ld;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(ldm<RES>(ok + j), vk[j - NX], acc);
  }
  if (k < N) {
    const float *ok1 = Mo + (int64_t)k * NX * ld + i;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(ldm<RES>(ok1 + j * ld), vk[NX + j], acc);
  }
  return acc;
}

template <int NX, int OP, int RED, bool RES>
__device__ void pcg_solve(const PcgArgs &a, int p, float *sm, typename Red<RED>::T *slots) {
  using R = Red<RED>;
  using AccT = typename R::T;
  const ProbDesc d = a.ps.get(p);
  const int N = d.N, n = N + 1, nu = d.nu, R_ = n * NX;
  const int tid = threadIdx.x, T = blockDim.x;
  const PcgLayout L = pcg_layout(OP, RES, N, NX, nu);
  float *sp = sm + L.p, *sr = sm + L.r, *sw = sm + L.w, *sv = sm + L.v;
  const float *gam = a.gamma + d.ovec;
  float *x = a.lambda + d.ovec;

  // ---- operator and preconditioner views ----
  const float *mA, *mB, *mIq, *mIr, *mD, *mE, *mPD, *mPE;
  const float *gq = a.qd + d.oq, *gr = a.rd + d.orr;
  int lda, ldb;
  if constexpr (RES) {
    lda = pad_ld(NX);
    ldb = pad_ld(nu > 0 ? nu : 1);
    float *s0 = sm + L.m0, *s1 = sm + L.m1, *spd = sm + L.pd, *spe = sm + L.pe;
    // stage once: global (dense, ld = NX) -> shared (padded ld)
    const float *gpd = a.PD + d.odiag, *gpe = a.PE + d.ooff;
    for (int e = tid; e < n * NX * NX; e += T) {
      const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
      spd[(b * NX + r) * lda + c] = gpd[e];
    }
    for (int e = tid; e < N * NX * NX; e += T) {
      const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
      spe[(b * NX + r) * lda + c] = gpe[e];
    }
    if constexpr (OP == kOpQp) {
      const float *gA = a.A + d.oA, *gB = a.B + d.oB;
      float *siq = sm + L.iq, *sir = sm + L.ir;
      for (int e = tid; e < N * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s0[(b * NX + r) * lda + c] = gA[e];
      }
      for (int e = tid; e < N * NX * nu; e += T) {
        const int row = e / nu, c = e - row * nu;
        s1[row * ldb + c] = gB[e];
      }
      for (int e = tid; e < n * NX; e += T) siq[e] = 1.0f / gq[e];
      for (int e = tid; e < N * nu; e += T) sir[e] = 1.0f / gr[e];
      mA = s0; mB = s1; mIq = siq; mIr = sir;
      mD = mE = nullptr;
    } else {
      const float *gD = a.D + d.odiag, *gE = a.E + d.ooff;
      for (int e = tid; e < n * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s0[(b * NX + r) * lda + c] = gD[e];
      }
      for (int e = tid; e < N * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s1[(b * NX + r) * lda + c] = gE[e];
      }
      mD = s0; mE = s1;
      mA = mB = mIq = mIr = nullptr;
    }
    mPD = spd; mPE = spe;
  } else {
    lda = NX;
    ldb = nu;
    mA = a.A + d.oA; mB = a.B + d.oB; mIq = nullptr; mIr = nullptr;
    mD = a.D + d.odiag; mE = a.E + d.ooff;
    mPD = a.PD + d.odiag; mPE = a.PE + d.ooff;
  }
  (void)mA; (void)mB; (void)mIq; (void)mIr; (void)mD; (void)mE; (void)gq; (void)gr;

  // 1/q_k[j] and 1/r_k[j]: staged reciprocals, or the same reciprocal formed on the fly.
  auto inv_q = [&](int e) -> float {
    if constexpr (RES) return mIq[e];
    else return 1.0f / __ldg(gq + e);
  };
  auto inv_r = [&](int e) -> float {
    if constexpr (RES) return mIr[e];
    else return 1.0f / __ldg(gr + e);
  };

  // w = S v (own rows); v must be complete in shared memory (src).
  // QP form: phase 1 writes sv = G^-1 C^T src, barrier, phase 2 forms the rows.
  auto apply_S_phase1 = [&](const float *src) {
    if constexpr (OP == kOpQp) {
      const int nvx = n * NX, nitems = nvx + N * nu;
      const float inv_nu = nu > 0 ? 1.0f / (float)nu : 0.0f;
      for (int it = tid; it < nitems; it += T) {
        if (it < nvx) {
          const int k = it / NX, j = it - k * NX;
          float acc = -src[it];
          if (k < N) {
            const float *Ak = mA + (int64_t)k * NX * lda + j;  // column j of A_k
            const float *pk1 = src + (k + 1) * NX;
#pragma unroll
            for (int l = 0; l < NX; ++l) acc = fmaf(ldm<RES>(Ak + l * lda), pk1[l], acc);
          }
          sv[it] = acc * inv_q(it);
        } else {
          const int t2 = it - nvx;
          const int k = (int)(((float)t2 + 0.5f) * inv_nu);
          const int j = t2 - k * nu;
          const float *Bk = mB + (int64_t)k * NX * ldb + j;  // column j of B_k
          const float *pk1 = src + (k + 1) * NX;
          float acc = 0.0f;
#pragma unroll
          for (int l = 0; l < NX; ++l) acc = fmaf(ldm<RES>(Bk + l * ldb), pk1[l], acc);
          sv[it] = acc * inv_r(t2);
        }
      }
      __syncthreads();
    }
  };
  auto apply_S_row = [&](const float *src, int k, int i) -> float {
    if constexpr (OP == kOpQp) {
      float acc = -sv[k * NX + i];
      if (k > 0) {
        const float *Ar = mA + (int64_t)(k - 1) * NX * lda + i * lda;  // row i of A_{k-1}
        const float *vx = sv + (k - 1) * NX;
#pragma unroll
        for (int j = 0; j < NX; ++j) acc = fmaf(ldm<RES>(Ar + j), vx[j], acc);
        const float *Br = mB + (int64_t)(k - 1) * NX * ldb + i * ldb;  // row i of B_{k-1}
        const float *vu = sv + n * NX + (k - 1) * nu;
        for (int j = 0; j < nu; ++j) acc = fmaf(ldm<RES>(Br + j), vu[j], acc);
      }
      return acc;
    } else {
      return bt_row<NX, RES>(mD, mE, lda, N, k, i, src);
    }
  };
  auto apply_P_row = [&](const float *src, int k, int i) -> float {
    return bt_row<NX, RES>(mPD, mPE, lda, N, k, i, src);
  };

  if (RES) __syncthreads();  // staged matrices visible

  // ---- r0 = gamma - S x0, z0 = Phi^-1 r0, p0 = z0 ----
  AccT g1[1] = {R::zero()};
  for (int row = tid; row < R_; row += T) {
    const float g = gam[row];
    g1[0] = R::fma(g1[0], g, g);
    sp[row] = a.warm ? x[row] : 0.0f;
  }
  block_sum<RED, 1>(g1, slots);  // contains a barrier: sp complete
  const float gg = R::tof(g1[0]);
  const float thresh = a.tol2 * gg;
  const int max_iter = a.max_iter > 0 ? a.max_iter : 10 * n * NX;
  if (gg == 0.0f) {
    for (int row = tid; row < R_; row += T) x[row] = 0.0f;
    if (tid == 0) { a.iters[p] = 0; a.relres[p] = 0.0; a.status[p] = kOk; }
    __syncthreads();
    return;
  }
  bool warm = a.warm != 0;
  if (warm) {
    apply_S_phase1(sp);
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      sr[row] = gam[row] - apply_S_row(sp, k, i);
    }
  } else {
    for (int row = tid; row < R_; row += T) { sr[row] = gam[row]; x[row] = 0.0f; }
  }
  __syncthreads();
  AccT s2[2];
  float rz, rr;
  for (int pass = 0; pass < 2; ++pass) {
    s2[0] = R::zero(); s2[1] = R::zero();
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      const float z = apply_P_row(sr, k, i);
      const float r = sr[row];
      sw[row] = z;
      s2[0] = R::fma(s2[0], r, z);
      s2[1] = R::fma(s2[1], r, r);
    }
    block_sum<RED, 2>(s2, slots + 64);
    rz = R::tof(s2[0]);
    rr = R::tof(s2[1]);
    // warm start with fallback: restart from zero if lambda_0 is no better than zero
    if (pass == 0 && warm && a.warm == 2 && !(rr < gg)) {
      for (int row = tid; row < R_; row += T) { sr[row] = gam[row]; x[row] = 0.0f; }
      warm = false;
      __syncthreads();
      continue;
    }
    break;
  }
  for (int row = tid; row < R_; row += T) sp[row] = sw[row];
  __syncthreads();

  // ---- iterations ----
  int it = 0, code = kOk;
  while (true) {
    if (!(rr > thresh)) {
      if (!isfinite(rr)) code = kNonFinite;
      break;
    }
    if (it >= max_iter) { code = kMaxIter; break; }
    // w = S p, p.w
    apply_S_phase1(sp);
    AccT s1[1] = {R::zero()};
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      const float w = apply_S_row(sp, k, i);
      sw[row] = w;
      s1[0] = R::fma(s1[0], sp[row], w);
    }
    block_sum<RED, 1>(s1, slots);
    const float pw = R::tof(s1[0]);
    if (!(pw > 0.0f) || !isfinite(pw)) { code = isfinite(pw) ? kBreakdown : kNonFinite; break; }
    const float alpha = rz / pw;
    for (int row = tid; row < R_; row += T) {
      x[row] = fmaf(alpha, sp[row], x[row]);
      sr[row] = fmaf(-alpha, sw[row], sr[row]);
    }
    __syncthreads();
    // z = Phi^-1 r, r.z, r.r
    s2[0] = R::zero(); s2[1] = R::zero();
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      const float z = apply_P_row(sr, k, i);
      const float r = sr[row];
      sw[row] = z;
      s2[0] = R::fma(s2[0], r, z);
      s2[1] = R::fma(s2[1], r, r);
    }
    block_sum<RED, 2>(s2, slots + 64);
    const float rz_new = R::tof(s2[0]);
    rr = R::tof(s2[1]);
    const float beta = rz_new / rz;
    rz = rz_new;
    for (int row = tid; row < R_; row += T) sp[row] = fmaf(beta, sp[row], sw[row]);
    __syncthreads();
    ++it;
  }
  if (tid == 0) {
    a.iters[p] = it;
    a.relres[p] = sqrt((double)rr / (double)gg);
    a.status[p] = code;
  }
  __syncthreads();
}

// Persistent kernel: CTAs take problems from the work list, through an
// atomic counter when one is given (largest problems first), else by stride.
template <int NX, int OP, int RED, bool RES>
__global__ void __launch_bounds__(512) pcg_kernel(PcgArgs a) {
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  __shared__ __align__(16) typename Red<RED>::T slots[4 * 32];
  __shared__ int s_next;
  int stride_i = 0;
  while (true) {
    int w;
    if (a.counter) {
      if (threadIdx.x == 0) s_next = atomicAdd(a.counter, 1);
      __syncthreads();
      w = s_next;
      __syncthreads();
    } else {
      w = blockIdx.x + stride_i * gridDim.x;
      ++stride_i;
    }
    if (w >= a.nwork) break;
    const int p = a.work ? a.work[w] : w;
    if (a.status[p] != kOk) continue;  // preconditioner failed for this problem
    pcg_solve<NX, OP, RED, RES>(a, p, sm, slots);
  }
}

}  // namespace sspcg

// Instantiate every kernel variant for one nx and register a launcher.
#define SSPCG_INSTANTIATE_PCG(NXV)                                                                      \
  namespace sspcg {                                                                                     \
  template <int OP, int RED, bool RES>                                                                  \
  static cudaError_t launch_one_##NXV(const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st) { \
    auto k = pcg_kernel<NXV, OP, RED, RES>;                                                             \
    static bool attr = false;                                                                           \
    if (!attr) {                                                                                        \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, pcg_max_smem_bytes()); \
      if (e != cudaSuccess) return e;                                                                   \
      attr = true;                                                                                      \
    }                                                                                                   \
    k<<<grid, block, smem, st>>>(a);                                                                    \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_pcg_nx##NXV(int op, int red, bool res, const PcgArgs &a, int grid, int block, size_t smem, \
                                 cudaStream_t st) {                                                     \
    if (op == kOpQp) {                                                                                  \
      if (red == kRedF32) return res ? launch_one_##NXV<kOpQp, kRedF32, true>(a, grid, block, smem, st)  \
                                     : launch_one_##NXV<kOpQp, kRedF32, false>(a, grid, block, smem, st); \
      if (red == kRedDf) return res ? launch_one_##NXV<kOpQp, kRedDf, true>(a, grid, block, smem, st)    \
                                    : launch_one_##NXV<kOpQp, kRedDf, false>(a, grid, block, smem, st);  \
      return res ? launch_one_##NXV<kOpQp, kRedF64, true>(a, grid, block, smem, st)                     \
                 : launch_one_##NXV<kOpQp, kRedF64, false>(a, grid, block, smem, st);                   \
    }                                                                                                   \
    if (red == kRedF32) return res ? launch_one_##NXV<kOpBlock, kRedF32, true>(a, grid, block, smem, st) \
                                   : launch_one_##NXV<kOpBlock, kRedF32, false>(a, grid, block, smem, st); \
    if (red == kRedDf) return res ? launch_one_##NXV<kOpBlock, kRedDf, true>(a, grid, block, smem, st)   \
                                  : launch_one_##NXV<kOpBlock, kRedDf, false>(a, grid, block, smem, st); \
    return res ? launch_one_##NXV<kOpBlock, kRedF64, true>(a, grid, block, smem, st)                    \
               : launch_one_##NXV<kOpBlock, kRedF64, false>(a, grid, block, smem, st);                  \
  }                                                                                                     \
  }
