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

// bt_row from global memory with every access by column: the sub-diagonal
// block's row i is read as column i of its transpose (Mot), so consecutive
// rows i of a warp read consecutive addresses.
template <int NX, typename Real, typename MT>
__device__ __forceinline__ Real bt_row_t(const MT *Md, const MT *Mo, const MT *Mot, int N, int k, int i,
                                         const Real *v) {
  const Real *vk = v + k * NX;
  const MT *dk = Md + (int64_t)k * NX * NX + i;
  Real acc = Real(0);
#pragma unroll
  for (int j = 0; j < NX; ++j) acc = rfma((Real)__ldg(dk + j * NX), vk[j], acc);
  if (k > 0) {
    const MT *ok = Mot + (int64_t)(k - 1) * NX * NX + i;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = rfma((Real)__ldg(ok + j * NX), vk[j - NX], acc);
  }
  if (k < N) {
    const MT *ok1 = Mo + (int64_t)k * NX * NX + i;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = rfma((Real)__ldg(ok1 + j * NX), vk[NX + j], acc);
  }
  return acc;
}

template <int NX, typename Real>
__device__ __forceinline__ void stage_blocks(Real *dst, const Real *src, int nblk, int ld, int tid, int T) {
  for (int e = tid; e < nblk * NX * NX; e += T) {
    const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
    dst[(b * NX + r) * ld + c] = src[e];
  }
}

// Operator and preconditioner blocks of one problem: the first K block rows
// staged in shared memory (odd row strides), the rest read from global
// memory (dense, row stride nx) through L1/L2.  Row k < K uses the staged
// copies only (its off-diagonal slots k-1 and k are staged with it).
template <typename Real>
struct Views {
  const Real *sA, *sB, *sD, *sE, *sPD, *sPE;      // staged (shared memory)
  const float *gA, *gB, *gD, *gE;                 // FP32 inputs (global)
  const Real *gPD, *gPE;                          // preconditioner (global)
  const float *gAt, *gBt;                         // transposed A_k, B_k (global, optional)
  const Real *gPEt;                               // transposed PE blocks (global, optional)
  int ld, ldb;                                    // staged row strides
};

template <int NX, int OP, int RED, typename Real>
__device__ void pcg_solve(const PcgArgs &a, const ProbDesc &d, Real *sm, typename Red<RED, Real>::T *slots) {
  using R = Red<RED, Real>;
  using AccT = typename R::T;
  const int p = d.id;  // output slot
  const int N = d.N, n = N + 1, nu = d.nu, R_ = n * NX;
  const int tid = threadIdx.x, T = blockDim.x;
  int K = pcg_max_resident(OP, N, NX, nu, a.smem_elems);  // the host sized smem so that K >= 0
  if (K > a.max_resident) K = a.max_resident;
  if (K < 0) K = 0;
  const int Ks = K < N ? K : N;
  const PcgLayout L = pcg_layout(OP, K, N, NX, nu);
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

  // ---- views and staging ----
  Views<Real> V{};
  V.ld = pad_ld(NX);
  V.ldb = pad_ld(nu > 0 ? nu : 1);
  V.gPD = reinterpret_cast<const Real *>(a.PD) + d.odiag;
  V.gPE = reinterpret_cast<const Real *>(a.PE) + d.ooff;
  V.gPEt = a.PEt ? reinterpret_cast<const Real *>(a.PEt) + d.ooff : nullptr;
  {
    Real *spd = sm + L.pd, *spe = sm + L.pe;
    stage_blocks<NX>(spd, V.gPD, K, V.ld, tid, T);
    stage_blocks<NX>(spe, V.gPE, Ks, V.ld, tid, T);
    V.sPD = spd; V.sPE = spe;
  }
  const float *gq = a.qd + d.oq, *gr = a.rd + d.orr;
  Real *siq = sm + L.iq, *sir = sm + L.ir;
  if constexpr (OP == kOpQp) {
    V.gA = a.A + d.oA;
    V.gB = a.B + d.oB;
    V.gAt = a.At ? a.At + d.oA : nullptr;
    V.gBt = a.Bt ? a.Bt + d.oB : nullptr;
    Real *s0 = sm + L.m0, *s1 = sm + L.m1;
    for (int e = tid; e < Ks * NX * NX; e += T) {
      const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
      s0[(b * NX + r) * V.ld + c] = (Real)V.gA[e];
    }
    for (int e = tid; e < Ks * NX * nu; e += T) {
      const int row = e / nu, c = e - row * nu;
      s1[row * V.ldb + c] = (Real)V.gB[e];
    }
    for (int e = tid; e < n * NX; e += T) siq[e] = Real(1) / (Real)gq[e];
    for (int e = tid; e < N * nu; e += T) sir[e] = Real(1) / (Real)gr[e];
    V.sA = s0; V.sB = s1;
  } else {
    V.gD = a.D + d.odiag;
    V.gE = a.E + d.ooff;
    Real *s0 = sm + L.m0, *s1 = sm + L.m1;
    for (int e = tid; e < K * NX * NX; e += T) {
      const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
      s0[(b * NX + r) * V.ld + c] = (Real)V.gD[e];
    }
    for (int e = tid; e < Ks * NX * NX; e += T) {
      const int b = e / (NX * NX), rem = e - b * NX * NX, r = rem / NX, c = rem - r * NX;
      s1[(b * NX + r) * V.ld + c] = (Real)V.gE[e];
    }
    V.sD = s0; V.sE = s1;
  }

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
            const Real *pk1 = src + (k + 1) * NX;
            if (k < K) {
              const Real *Ak = V.sA + k * NX * V.ld + j;  // column j of A_k (staged)
#pragma unroll
              for (int l = 0; l < NX; ++l) acc = rfma(Ak[l * V.ld], pk1[l], acc);
            } else {
              const float *Ak = V.gA + (int64_t)k * NX * NX + j;
#pragma unroll
              for (int l = 0; l < NX; ++l) acc = rfma((Real)__ldg(Ak + l * NX), pk1[l], acc);
            }
          }
          sv[it] = acc * siq[it];
        } else {
          const int t2 = it - nvx;
          const int k = (int)(((float)t2 + 0.5f) * inv_nu);
          const int j = t2 - k * nu;
          const Real *pk1 = src + (k + 1) * NX;
          Real acc = Real(0);
          if (k < K) {
            const Real *Bk = V.sB + k * NX * V.ldb + j;  // column j of B_k (staged)
#pragma unroll
            for (int l = 0; l < NX; ++l) acc = rfma(Bk[l * V.ldb], pk1[l], acc);
          } else {
            const float *Bk = V.gB + (int64_t)k * NX * nu + j;
#pragma unroll
            for (int l = 0; l < NX; ++l) acc = rfma((Real)__ldg(Bk + l * nu), pk1[l], acc);
          }
          sv[it] = acc * sir[t2];
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
        const Real *vx = sv + (k - 1) * NX;
        const Real *vu = sv + n * NX + (k - 1) * nu;
        if (k < K) {
          const Real *Ar = V.sA + ((k - 1) * NX + i) * V.ld;  // row i of A_{k-1}
#pragma unroll
          for (int j = 0; j < NX; ++j) acc = rfma(Ar[j], vx[j], acc);
          const Real *Br = V.sB + ((k - 1) * NX + i) * V.ldb;
          for (int j = 0; j < nu; ++j) acc = rfma(Br[j], vu[j], acc);
        } else if (V.gAt) {
          // row i of A_{k-1} = column i of its transpose: consecutive i are consecutive addresses
          const float *Ac = V.gAt + (int64_t)(k - 1) * NX * NX + i;
#pragma unroll
          for (int j = 0; j < NX; ++j) acc = rfma((Real)__ldg(Ac + j * NX), vx[j], acc);
          const float *Bc = V.gBt + (int64_t)(k - 1) * nu * NX + i;
          for (int j = 0; j < nu; ++j) acc = rfma((Real)__ldg(Bc + j * NX), vu[j], acc);
        } else {
          const float *Ar = V.gA + ((int64_t)(k - 1) * NX + i) * NX;
#pragma unroll
          for (int j = 0; j < NX; ++j) acc = rfma((Real)__ldg(Ar + j), vx[j], acc);
          const float *Br = V.gB + ((int64_t)(k - 1) * NX + i) * nu;
          for (int j = 0; j < nu; ++j) acc = rfma((Real)__ldg(Br + j), vu[j], acc);
        }
      }
      return acc;
    } else {
      return k < K ? bt_row<NX, true, Real>(V.sD, V.sE, V.ld, N, k, i, src)
                   : bt_row<NX, false, Real>(V.gD, V.gE, NX, N, k, i, src);
    }
  };
  auto apply_P_row = [&](const Real *src, int k, int i) -> Real {
    if (k < K) return bt_row<NX, true, Real>(V.sPD, V.sPE, V.ld, N, k, i, src);
    if (V.gPEt) return bt_row_t<NX, Real>(V.gPD, V.gPE, V.gPEt, N, k, i, src);
    return bt_row<NX, false, Real>(V.gPD, V.gPE, NX, N, k, i, src);
  };

  __syncthreads();  // staged blocks and reciprocals visible

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
template <int NX, int OP, int RED, typename Real>
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
    pcg_solve<NX, OP, RED, Real>(a, d, sm, slots);
  }
}

template <int NX, int OP, int RED, typename Real>
cudaError_t launch_variant(const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
  auto k = pcg_kernel<NX, OP, RED, Real>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, pcg_max_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  PcgArgs b = a;
  b.smem_elems = (int64_t)(smem / sizeof(Real));
  k<<<grid, block, smem, st>>>(b);
  return cudaGetLastError();
}

// All variants of one nx: FP32 with three reduction modes for both operator
// forms, and the FP64 path (QP form, FP64 reductions).
template <int NX>
cudaError_t launch_pcg_for_nx(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem,
                              cudaStream_t st) {
  if (f64) {
    if (op != kOpQp) return cudaErrorInvalidValue;
    return launch_variant<NX, kOpQp, kRedF64, double>(a, grid, block, smem, st);
  }
#define SSPCG_PCG_CASE(OPV, REDV) \
  if (op == OPV && red == REDV) return launch_variant<NX, OPV, REDV, float>(a, grid, block, smem, st);
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
  cudaError_t launch_pcg_nx##NXV(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, \
                                 cudaStream_t st) {                                                          \
    return launch_pcg_for_nx<NXV>(op, red, f64, a, grid, block, smem, st);                                    \
  }                                                                                                          \
  }
