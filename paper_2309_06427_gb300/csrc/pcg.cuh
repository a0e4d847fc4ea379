// Fused PCG kernel: one CTA runs the whole preconditioned CG loop of one
// problem (Sec. II-B), with S p and Phi^-1 r as block-tridiagonal products
// and the dot products reduced by warp shuffles.  Included by the per-nx
// instantiation units.
//
// Thread mapping: thread t owns rows t, t + T, t + 2T, ... of the
// (N+1)*nx unknowns; row = k*nx + i is row i of block row k.
//
// Per iteration (textbook PCG, Saad Alg. 9.1):
//   w = S p                 (QP form: v = G^-1 C^T p, barrier, w = C v)
//   alpha = (r.z) / (p.w)   block reduction
//   x += alpha p, r -= alpha w, barrier
//   z = Phi^-1 r, (r.z), (r.r) block reduction
//   beta = (r.z)new / (r.z)old, p = z + beta p, barrier
// Stop before an iteration once r.r <= tol^2 gamma.gamma.
//
// Real is the working precision (float: the fast path; double: the FP64
// path).  The QP data A, B, diag Q, diag R and gamma are FP32 inputs in both
// and are converted exactly; Phi^-1 blocks, vectors and lambda are Real.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace sspcg {

__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }

template <bool RES, typename T>
__device__ __forceinline__ T ldm(const T *p) {
  if constexpr (RES) return *p;
  else return __ldg(p);
}

// Accumulators of the reduction modes.
template <int RED, typename Real> struct Red;
template <> struct Red<kRedF32, float> {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.0f; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return fmaf(a, b, acc); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float get(T v) { return v; }
};
template <> struct Red<kRedDf, float> {
  using T = df;
  static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return df_fma(acc, a, b); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float get(T v) { return __fadd_rn(v.hi, v.lo); }
};
template <> struct Red<kRedF64, float> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T fma(T acc, float a, float b) { return ::fma((double)a, (double)b, acc); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ float get(T v) { return (float)v; }
};
template <> struct Red<kRedF64, double> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T fma(T acc, double a, double b) { return ::fma(a, b, acc); }
  static __device__ __forceinline__ T sum(T v) { return warp_sum(v); }
  static __device__ __forceinline__ double get(T v) { return v; }
};

// Block-wide sum of K accumulators: warp butterflies, one slot per warp,
// one barrier, then every warp sums the slots in the same order, so all
// threads hold bit-identical results.
template <class R, int K>
__device__ __forceinline__ void block_sum(typename R::T (&v)[K], typename R::T *slots) {
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
template <int NX, bool RES, typename Real, typename MT>
__device__ __forceinline__ Real bt_row(const MT *Md, const MT *Mo, int ld, int N, int k, int i, const Real *v) {
  const Real *vk = v + k * NX;
  const MT *dk = Md + (int64_t)k * NX * ld + i;
  Real acc = Real(0);
#pragma unroll
  for (int j = 0; j < NX; ++j) acc = rfma((Real)ldm<RES>(dk + j * ld), vk[j], acc);
  if (k > 0) {
    const MT *ok = Mo + (int64_t)(k - 1) * NX * ld + i * ld;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = rfma((Real)ldm<RES>(ok + j), vk[j - NX], acc);
  }
  if (k < N) {
    const MT *ok1 = Mo + (int64_t)k * NX * ld + i;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = rfma((Real)ldm<RES>(ok1 + j * ld), vk[NX + j], acc);
  }
  return acc;
}

template <int NX, bool RES, typename Real, typename ST>
__device__ __forceinline__ void stage_blocks(ST *dst, const ST *src, int nblk, int ld, int tid, int T) {
  for (int e = tid; e < nblk * NX * NX; e += T) {
    const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
    dst[(b * NX + r) * ld + c] = src[e];
  }
}

template <int NX, int OP, int RED, bool RES, typename Real>
__device__ void pcg_solve(const PcgArgs &a, const ProbDesc &d, Real *sm, typename Red<RED, Real>::T *slots) {
  using R = Red<RED, Real>;
  using AccT = typename R::T;
  // operator matrices: staged as Real in shared memory, or FP32 from global memory
  using OpT = std::conditional_t<RES, Real, float>;
  const int p = d.id;  // output slot
  const int N = d.N, n = N + 1, nu = d.nu, R_ = n * NX;
  const int tid = threadIdx.x, T = blockDim.x;
  const PcgLayout L = pcg_layout(OP, RES, N, NX, nu);
  Real *sp = sm + L.p, *sr = sm + L.r, *sw = sm + L.w, *sx = sm + L.x, *sv = sm + L.v;
  const float *gam = a.gamma + d.ovec;
  // lambda (global): read once for a warm start, written once at the end
  auto lam_load = [&](int row) -> Real {
    if (a.lambda_f32) return (Real) reinterpret_cast<const float *>(a.lambda)[d.ovec + row];
    return reinterpret_cast<const Real *>(a.lambda)[d.ovec + row];
  };
  auto lam_store = [&](int row, Real v) {
    if (a.lambda_f32) reinterpret_cast<float *>(a.lambda)[d.ovec + row] = (float)v;
    else reinterpret_cast<Real *>(a.lambda)[d.ovec + row] = v;
  };
  const Real *gPD = reinterpret_cast<const Real *>(a.PD) + d.odiag;
  const Real *gPE = reinterpret_cast<const Real *>(a.PE) + d.ooff;

  // ---- operator and preconditioner views ----
  const OpT *mA = nullptr, *mB = nullptr, *mD = nullptr, *mE = nullptr;
  const Real *mIq = nullptr, *mIr = nullptr, *mPD, *mPE;
  const float *gq = a.qd + d.oq, *gr = a.rd + d.orr;
  int lda, ldb;
  if constexpr (RES) {
    lda = pad_ld(NX);
    ldb = pad_ld(nu > 0 ? nu : 1);
    Real *s0 = sm + L.m0, *s1 = sm + L.m1, *spd = sm + L.pd, *spe = sm + L.pe;
    stage_blocks<NX, RES, Real>(spd, gPD, n, lda, tid, T);
    stage_blocks<NX, RES, Real>(spe, gPE, N, lda, tid, T);
    if constexpr (OP == kOpQp) {
      const float *gA = a.A + d.oA, *gB = a.B + d.oB;
      Real *siq = sm + L.iq, *sir = sm + L.ir;
      for (int e = tid; e < N * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s0[(b * NX + r) * lda + c] = (Real)gA[e];
      }
      for (int e = tid; e < N * NX * nu; e += T) {
        const int row = e / nu, c = e - row * nu;
        s1[row * ldb + c] = (Real)gB[e];
      }
      for (int e = tid; e < n * NX; e += T) siq[e] = Real(1) / (Real)gq[e];
      for (int e = tid; e < N * nu; e += T) sir[e] = Real(1) / (Real)gr[e];
      mA = s0; mB = s1; mIq = siq; mIr = sir;
    } else {
      const float *gD = a.D + d.odiag, *gE = a.E + d.ooff;
      for (int e = tid; e < n * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s0[(b * NX + r) * lda + c] = (Real)gD[e];
      }
      for (int e = tid; e < N * NX * NX; e += T) {
        const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
        s1[(b * NX + r) * lda + c] = (Real)gE[e];
      }
      mD = s0; mE = s1;
    }
    mPD = spd; mPE = spe;
  } else {
    lda = NX;
    ldb = nu;
    if constexpr (OP == kOpQp) { mA = a.A + d.oA; mB = a.B + d.oB; }
    else { mD = a.D + d.odiag; mE = a.E + d.ooff; }
    mPD = gPD; mPE = gPE;
  }

  // 1/q_k[j] and 1/r_k[j]: staged reciprocals, or the same reciprocal formed on the fly.
  auto inv_q = [&](int e) -> Real {
    if constexpr (RES) return mIq[e];
    else return Real(1) / (Real)__ldg(gq + e);
  };
  auto inv_r = [&](int e) -> Real {
    if constexpr (RES) return mIr[e];
    else return Real(1) / (Real)__ldg(gr + e);
  };

  // QP form, phase 1: sv = G^-1 C^T src (all threads), then a barrier.
  auto apply_S_phase1 = [&](const Real *src) {
    if constexpr (OP == kOpQp) {
      const int nvx = n * NX, nitems = nvx + N * nu;
      const float inv_nu = nu > 0 ? 1.0f / (float)nu : 0.0f;
      for (int it = tid; it < nitems; it += T) {
        if (it < nvx) {
          const int k = it / NX, j = it - k * NX;
          Real acc = -src[it];
          if (k < N) {
            const OpT *Ak = mA + (int64_t)k * NX * lda + j;  // column j of A_k
            const Real *pk1 = src + (k + 1) * NX;
#pragma unroll
            for (int l = 0; l < NX; ++l) acc = rfma((Real)ldm<RES>(Ak + l * lda), pk1[l], acc);
          }
          sv[it] = acc * inv_q(it);
        } else {
          const int t2 = it - nvx;
          const int k = (int)(((float)t2 + 0.5f) * inv_nu);
          const int j = t2 - k * nu;
          const OpT *Bk = mB + (int64_t)k * NX * ldb + j;  // column j of B_k
          const Real *pk1 = src + (k + 1) * NX;
          Real acc = Real(0);
#pragma unroll
          for (int l = 0; l < NX; ++l) acc = rfma((Real)ldm<RES>(Bk + l * ldb), pk1[l], acc);
          sv[it] = acc * inv_r(t2);
        }
      }
      __syncthreads();
    }
  };
  // Row (k, i) of S src (QP form: of C sv).
  auto apply_S_row = [&](const Real *src, int k, int i) -> Real {
    if constexpr (OP == kOpQp) {
      Real acc = -sv[k * NX + i];
      if (k > 0) {
        const OpT *Ar = mA + (int64_t)(k - 1) * NX * lda + i * lda;  // row i of A_{k-1}
        const Real *vx = sv + (k - 1) * NX;
#pragma unroll
        for (int j = 0; j < NX; ++j) acc = rfma((Real)ldm<RES>(Ar + j), vx[j], acc);
        const OpT *Br = mB + (int64_t)(k - 1) * NX * ldb + i * ldb;  // row i of B_{k-1}
        const Real *vu = sv + n * NX + (k - 1) * nu;
        for (int j = 0; j < nu; ++j) acc = rfma((Real)ldm<RES>(Br + j), vu[j], acc);
      }
      return acc;
    } else {
      return bt_row<NX, RES, Real>(mD, mE, lda, N, k, i, src);
    }
  };
  auto apply_P_row = [&](const Real *src, int k, int i) -> Real {
    return bt_row<NX, RES, Real>(mPD, mPE, lda, N, k, i, src);
  };

  if (RES) __syncthreads();  // staged matrices visible

  // ---- r0 = gamma - S x0, z0 = Phi^-1 r0, p0 = z0 ----
  AccT g1[1] = {R::zero()};
  for (int row = tid; row < R_; row += T) {
    const Real g = (Real)gam[row];
    g1[0] = R::fma(g1[0], g, g);
    const Real x0 = a.warm ? lam_load(row) : Real(0);
    sp[row] = x0;
    sx[row] = x0;
  }
  block_sum<R, 1>(g1, slots);  // contains a barrier: sp complete
  const Real gg = R::get(g1[0]);
  const Real thresh = (Real)a.tol2 * gg;
  const int max_iter = a.max_iter > 0 ? a.max_iter : 10 * n * NX;
  if (gg == Real(0)) {
    for (int row = tid; row < R_; row += T) lam_store(row, Real(0));
    if (tid == 0) { a.iters[p] = 0; a.relres[p] = 0.0; a.status[p] = kOk; }
    __syncthreads();
    return;
  }
  bool warm = a.warm != 0;
  if (warm) {
    apply_S_phase1(sp);
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      sr[row] = (Real)gam[row] - apply_S_row(sp, k, i);
    }
  } else {
    for (int row = tid; row < R_; row += T) sr[row] = (Real)gam[row];
  }
  __syncthreads();
  AccT s2[2];
  Real rz, rr;
  for (int pass = 0; pass < 2; ++pass) {
    s2[0] = R::zero(); s2[1] = R::zero();
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      const Real z = apply_P_row(sr, k, i);
      const Real r = sr[row];
      sw[row] = z;
      s2[0] = R::fma(s2[0], r, z);
      s2[1] = R::fma(s2[1], r, r);
    }
    block_sum<R, 2>(s2, slots + 64);
    rz = R::get(s2[0]);
    rr = R::get(s2[1]);
    // warm start with fallback: restart from zero if lambda_0 is no better than zero
    if (pass == 0 && warm && a.warm == 2 && !(rr < gg)) {
      for (int row = tid; row < R_; row += T) { sr[row] = (Real)gam[row]; sx[row] = Real(0); }
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
      const Real w = apply_S_row(sp, k, i);
      sw[row] = w;
      s1[0] = R::fma(s1[0], sp[row], w);
    }
    block_sum<R, 1>(s1, slots);
    const Real pw = R::get(s1[0]);
    if (!(pw > Real(0)) || !isfinite(pw)) { code = isfinite(pw) ? kBreakdown : kNonFinite; break; }
    const Real alpha = rz / pw;
    for (int row = tid; row < R_; row += T) {
      sx[row] = rfma(alpha, sp[row], sx[row]);
      sr[row] = rfma(-alpha, sw[row], sr[row]);
    }
    __syncthreads();
    // z = Phi^-1 r, r.z, r.r
    s2[0] = R::zero(); s2[1] = R::zero();
    for (int row = tid; row < R_; row += T) {
      const int k = row / NX, i = row - k * NX;
      const Real z = apply_P_row(sr, k, i);
      const Real r = sr[row];
      sw[row] = z;
      s2[0] = R::fma(s2[0], r, z);
      s2[1] = R::fma(s2[1], r, r);
    }
    block_sum<R, 2>(s2, slots + 64);
    const Real rz_new = R::get(s2[0]);
    rr = R::get(s2[1]);
    const Real beta = rz_new / rz;
    rz = rz_new;
    for (int row = tid; row < R_; row += T) sp[row] = rfma(beta, sp[row], sw[row]);
    __syncthreads();
    ++it;
  }
  for (int row = tid; row < R_; row += T) lam_store(row, sx[row]);
  if (tid == 0) {
    a.iters[p] = it;
    a.relres[p] = sqrt((double)rr / (double)gg);
    a.status[p] = code;
  }
  __syncthreads();
}

// Persistent kernel: CTAs take problems from the work list, through an
// atomic counter when one is given (largest problems first), else by stride.
template <int NX, int OP, int RED, bool RES, typename Real>
__global__ void __launch_bounds__(512) pcg_kernel(PcgArgs a) {
  extern __shared__ float4 smem4[];
  Real *sm = reinterpret_cast<Real *>(smem4);
  __shared__ __align__(16) typename Red<RED, Real>::T slots[4 * 32];
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
    const ProbDesc d = a.ps.get(a.work ? a.work[w] : w);
    if (a.status[d.id] != kOk) continue;  // preconditioner failed for this problem
    pcg_solve<NX, OP, RED, RES, Real>(a, d, sm, slots);
  }
}

template <int NX, int OP, int RED, bool RES, typename Real>
cudaError_t launch_variant(const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
  auto k = pcg_kernel<NX, OP, RED, RES, Real>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, pcg_max_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// All variants of one nx: FP32 with three reduction modes for both operator
// forms and both schedules, and the FP64 path (QP form, FP64 reductions).
template <int NX>
cudaError_t launch_pcg_for_nx(int op, int red, bool res, bool f64, const PcgArgs &a, int grid, int block,
                              size_t smem, cudaStream_t st) {
  if (f64) {
    if (op != kOpQp) return cudaErrorInvalidValue;
    return res ? launch_variant<NX, kOpQp, kRedF64, true, double>(a, grid, block, smem, st)
               : launch_variant<NX, kOpQp, kRedF64, false, double>(a, grid, block, smem, st);
  }
#define SSPCG_PCG_CASE(OPV, REDV)                                                   \
  if (op == OPV && red == REDV)                                                     \
    return res ? launch_variant<NX, OPV, REDV, true, float>(a, grid, block, smem, st) \
               : launch_variant<NX, OPV, REDV, false, float>(a, grid, block, smem, st);
  SSPCG_PCG_CASE(kOpQp, kRedDf)
  SSPCG_PCG_CASE(kOpQp, kRedF32)
  SSPCG_PCG_CASE(kOpQp, kRedF64)
  SSPCG_PCG_CASE(kOpBlock, kRedDf)
  SSPCG_PCG_CASE(kOpBlock, kRedF32)
  SSPCG_PCG_CASE(kOpBlock, kRedF64)
#undef SSPCG_PCG_CASE
  return cudaErrorInvalidValue;
}

}  // namespace sspcg

#define SSPCG_INSTANTIATE_PCG(NXV)                                                                           \
  namespace sspcg {                                                                                          \
  cudaError_t launch_pcg_nx##NXV(int op, int red, bool res, bool f64, const PcgArgs &a, int grid, int block, \
                                 size_t smem, cudaStream_t st) {                                             \
    return launch_pcg_for_nx<NXV>(op, red, res, f64, a, grid, block, smem, st);                               \
  }                                                                                                          \
  }
