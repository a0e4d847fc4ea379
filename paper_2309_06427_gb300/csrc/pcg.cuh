// Fused PCG kernel: one CTA runs the whole preconditioned CG loop of one
// problem (Sec. II-B), with S p and Phi^-1 r as block-tridiagonal products
// and the dot products reduced by warp shuffles.  Included by the per-nx
// instantiation units.
//
// Thread mapping: thread t owns rows t, t + T, t + 2T, ... of the
// (N+1)*nx unknowns; row = k*nx + i is row i of block row k.  Vectors live
// in shared memory with a block-row stride of nx rounded up to 4, and each
// row loads the block-row segments it multiplies into registers with
// 128-bit loads.
//
// Per iteration (textbook PCG, Saad Alg. 9.1):
//   w = S p                 (QP form: v = G^-1 C^T p, barrier, w = C v)
//   alpha = (r.z) / (p.w)   block reduction
//   x += alpha p, r -= alpha w, barrier
//   z = Phi^-1 r, (r.z), (r.r) block reduction
//     (degree-d polynomial preconditioner: z = Phi^-1 r, then d times
//      e = S-residual r - S z, barrier, z += Phi^-1 e; the sums after the last)
//   beta = (r.z)new / (r.z)old, p = z + beta p, barrier
// Stop before an iteration once r.r <= tol^2 gamma.gamma.
// The CG template flag selects the single-reduction form of the same
// iteration (Chronopoulos & Gear): s = S p by recurrence, one block sum of
// (r.u, S u.u, r.r) per iteration; see the CG section of pcg_solve.
//
// The first K block rows of the operator and preconditioner blocks are
// staged in shared memory (odd row strides); the rest are read from global
// memory every iteration (L1/L2).  Problems whose vectors alone exceed the
// shared memory keep them in a per-CTA slot of a global workspace (K = 0).
//
// Real is the working precision (float: the fast path; double: the FP64
// path).  The QP data A, B, diag Q, diag R and gamma are FP32 inputs in both
// and are converted exactly; Phi^-1 blocks, vectors and lambda are Real.
#pragma once

#include <cstring>
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

// Pieces of the reductions for every accumulator type: the sum of two partial sums (double-float: TwoSum,
// exact in its high and low parts, and the same whichever operand comes first), and warp shuffles.
__device__ __forceinline__ float red_add(float a, float b) { return a + b; }
__device__ __forceinline__ double red_add(double a, double b) { return a + b; }
__device__ __forceinline__ df red_add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ float red_shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double red_shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df red_shfl_xor(df v, int o) { return df_shfl_xor(v, o); }
__device__ __forceinline__ float red_shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double red_shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ df red_shfl(df v, int src) {
  return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// Xor butterfly over the 16 lanes of each half-warp.  The two lanes of a pair add the same two values, so
// every lane of a half ends with the same sum.
template <typename T>
__device__ __forceinline__ T half_warp_sum(T v) {
#pragma unroll
  for (int o = 8; o; o >>= 1) v = red_add(v, red_shfl_xor(v, o));
  return v;
}

// Warp sum of two accumulators with the work split between the half-warps (reduce-scatter): lanes 0-15 end
// with the sum of a, lanes 16-31 with the sum of b, each half identical across its lanes.  The first step
// trades across the halves (each lane sends the value its half does not keep), the other four run within a
// half on one value.
template <typename T>
__device__ __forceinline__ T warp_sum_split(T a, T b) {
  const bool hi = (threadIdx.x & 31) >= 16;
  const T keep = hi ? b : a, give = hi ? a : b;
  return half_warp_sum(red_add(keep, red_shfl_xor(give, 16)));
}

// Block-wide sum of K accumulators, every thread holding bit-identical results: warp sums, one slot per warp,
// one barrier, then every warp sums the slots (at most 16: CTAs have at most 512 threads) in the same order.
// Pairs of accumulators go through warp_sum_split, a single one through a full butterfly; the second stage
// reads the slots into both halves of the warp (or one half per accumulator of a pair) and sums them over a
// half-warp, then lanes 0 and 16 broadcast a pair's two sums.
template <class R, int K>
__device__ __forceinline__ void block_sum(typename R::T (&v)[K], typename R::T *slots) {
  using T = typename R::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int h = lane >> 4, l16 = lane & 15;
  constexpr int P = K / 2;  // pairs
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const T w = warp_sum_split(v[2 * q], v[2 * q + 1]);
    if (l16 == 0) slots[(2 * q + h) * 32 + wid] = w;
  }
  if constexpr (K % 2 == 1) {
    const T w = R::sum(v[K - 1]);
    if (lane == 0) slots[(K - 1) * 32 + wid] = w;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const T w = half_warp_sum(l16 < nw ? slots[(2 * q + h) * 32 + l16] : R::zero());
    v[2 * q] = red_shfl(w, 0);
    v[2 * q + 1] = red_shfl(w, 16);
  }
  if constexpr (K % 2 == 1) v[K - 1] = half_warp_sum(l16 < nw ? slots[(K - 1) * 32 + l16] : R::zero());
}

// The thread group that solves one problem: the CTA, or one warp (WARP: several problems per CTA, one per
// warp, with warp barriers and warp-only reductions).  A warp's xor butterfly leaves the same sum in every
// lane (each step adds the same two values in both lanes of a pair), so the scalars stay bit-identical across
// the group as in block_sum.
template <bool WARP>
__device__ __forceinline__ void group_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

template <class R, int K, bool WARP>
__device__ __forceinline__ void group_sum(typename R::T (&v)[K], typename R::T *slots) {
  if constexpr (WARP) {
    constexpr int P = K / 2;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const typename R::T w = warp_sum_split(v[2 * q], v[2 * q + 1]);
      v[2 * q] = red_shfl(w, 0);
      v[2 * q + 1] = red_shfl(w, 16);
    }
    if constexpr (K % 2 == 1) v[K - 1] = R::sum(v[K - 1]);
    __syncwarp();
  } else {
    block_sum<R, K>(v, slots);
  }
}

// A block-row segment of a vector in registers: NXP = nx rounded up to 4
// entries, loaded with 128-bit shared-memory loads (the segment starts
// 16-byte aligned; entries past nx are padding and never used).
template <int NX, typename Real>
struct Seg {
  static constexpr int NXP = (NX + 3) & ~3;
  Real v[NXP];
  __device__ __forceinline__ void load(const Real *src) {
    constexpr int per = 16 / (int)sizeof(Real);
#pragma unroll
    for (int q = 0; q < NXP / per; ++q) {
      const float4 c = reinterpret_cast<const float4 *>(src)[q];
      if constexpr (sizeof(Real) == 4) {
        v[4 * q + 0] = c.x; v[4 * q + 1] = c.y; v[4 * q + 2] = c.z; v[4 * q + 3] = c.w;
      } else {
        const double2 dd = *reinterpret_cast<const double2 *>(&c);
        v[2 * q + 0] = dd.x; v[2 * q + 1] = dd.y;
      }
    }
  }
};

// sum_{j < NX} m[j * stride] * seg[j] with two independent accumulators
// (even and odd j), so that consecutive FMAs do not wait on each other.
template <int NX, bool SMEM, typename Real, typename MT>
__device__ __forceinline__ Real dot_seg(const MT *m, int stride, const Real *seg) {
  Real a0 = Real(0), a1 = Real(0);
#pragma unroll
  for (int j = 0; j < NX; j += 2) {
    a0 = rfma((Real)ldm<SMEM>(m + j * stride), seg[j], a0);
    if (j + 1 < NX) a1 = rfma((Real)ldm<SMEM>(m + (j + 1) * stride), seg[j + 1], a1);
  }
  return a0 + a1;
}

// sum_{j < NX} m[j] * seg[j] for a 16-byte aligned row in global memory (the padded copies of streamed
// block rows), read through the read-only path with 128-bit loads (four FP32 or two FP64 values; entries past
// NX are padding and are not used); MT is the stored type.  The accumulation of dot_seg: even j into a0, odd
// j into a1, each in increasing j, so the result is bit-identical.
template <int NX, typename Real, typename MT>
__device__ __forceinline__ Real dot_row_g(const MT *m, const Real *seg) {
  constexpr int NXP = (NX + 3) & ~3;
  Real a0 = Real(0), a1 = Real(0);
  if constexpr (sizeof(MT) == 4 && NXP % 8 == 0) {
    // padded FP32 rows of a multiple of 8 values start 32-byte aligned (pad_region): 256-bit loads
#pragma unroll
    for (int q = 0; q < NXP / 8; ++q) {
      float c[8];
      asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]), "=f"(c[4]), "=f"(c[5]), "=f"(c[6]),
                     "=f"(c[7])
                   : "l"(m + 8 * q));
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = 8 * q + t;
        if (j < NX) {
          if (t % 2 == 0) a0 = rfma((Real)c[t], seg[j], a0);
          else a1 = rfma((Real)c[t], seg[j], a1);
        }
      }
    }
    return a0 + a1;
  }
#pragma unroll
  for (int q = 0; q < NXP * (int)sizeof(MT) / 16; ++q) {
    const float4 c = __ldg(reinterpret_cast<const float4 *>(m) + q);
    if constexpr (sizeof(MT) == 4) {
      const int j = 4 * q;
      if (j < NX) a0 = rfma((Real)c.x, seg[j], a0);
      if (j + 1 < NX) a1 = rfma((Real)c.y, seg[j + 1], a1);
      if (j + 2 < NX) a0 = rfma((Real)c.z, seg[j + 2], a0);
      if (j + 3 < NX) a1 = rfma((Real)c.w, seg[j + 3], a1);
    } else {
      const double2 dd = *reinterpret_cast<const double2 *>(&c);
      const int j = 2 * q;
      if (j < NX) a0 = rfma((Real)dd.x, seg[j], a0);
      if (j + 1 < NX) a1 = rfma((Real)dd.y, seg[j + 1], a1);
    }
  }
  return a0 + a1;
}

// Row (k, i) of the preconditioner for a streamed block row: PD dense (row stride NX, read by column), PE
// with row stride ldo; pad: PE rows are 16-byte aligned (the padded copy) and its sub-diagonal row is read
// with 128-bit loads.  The operation order of bt_row.
template <int NX, typename Real>
__device__ __forceinline__ Real bt_row_stream(const Real *Md, const Real *Mo, int ldo, bool pad, int N, int k, int i,
                                              const Real *v) {
  constexpr int NXP = (NX + 3) & ~3;
  Seg<NX, Real> s0, s1, s2;
  s0.load(v + k * NXP);
  s1.load(v + (k - 1) * NXP);
  s2.load(v + (k + 1) * NXP);
  const int km = k > 0 ? k - 1 : 0;
  const int kp = k < N ? k : (N > 0 ? N - 1 : 0);
  const Real a = dot_seg<NX, false, Real>(Md + (int64_t)k * NX * NX + i, NX, s0.v);
  const Real b = pad ? dot_row_g<NX, Real>(Mo + ((int64_t)km * NX + i) * ldo, s1.v)
                     : dot_seg<NX, false, Real>(Mo + ((int64_t)km * NX + i) * ldo, 1, s1.v);
  const Real c = dot_seg<NX, false, Real>(Mo + (int64_t)kp * NX * ldo + i, ldo, s2.v);
  return (a + b) + c;
}

// Row (k, i) of a block-tridiagonal symmetric matrix times v (block-row
// stride NXP): Md diagonal blocks (symmetric; read by column so that
// consecutive i are consecutive addresses), Mo sub-diagonal blocks with
// Mo[k-1] = M(k, k-1) (read by row), and M(k, k+1) = Mo[k]^T (read by
// column).  ld: row stride.  The segments of v at block rows -1 and N + 1
// are zero, so the three products run without branches and can overlap:
// the off-diagonal block index is clamped into range (slot 0, a zero block,
// when N = 0) and multiplies the zero segment at the ends.
template <int NX, bool SMEM, typename Real, typename MT>
__device__ __forceinline__ Real bt_row(const MT *Md, const MT *Mo, int ld, int N, int k, int i, const Real *v) {
  constexpr int NXP = (NX + 3) & ~3;
  Seg<NX, Real> s0, s1, s2;
  s0.load(v + k * NXP);
  s1.load(v + (k - 1) * NXP);
  s2.load(v + (k + 1) * NXP);
  const int km = k > 0 ? k - 1 : 0;
  const int kp = k < N ? k : (N > 0 ? N - 1 : 0);
  const Real a = dot_seg<NX, SMEM, Real>(Md + (int64_t)k * NX * ld + i, ld, s0.v);
  const Real b = dot_seg<NX, SMEM, Real>(Mo + ((int64_t)km * NX + i) * ld, 1, s1.v);
  const Real c = dot_seg<NX, SMEM, Real>(Mo + (int64_t)kp * NX * ld + i, ld, s2.v);
  return (a + b) + c;
}

// Staging: the first ``count`` elements of a dense row-major array with rows of width w (global) into shared
// memory rows of stride ld, converted to Real.  With a 16-byte aligned source (the packed layout aligns every
// problem's arrays) each thread takes 16 consecutive bytes per load (four FP32 or two FP64 values) and
// scatters them into the padded rows; the rest, or an unaligned source, one element at a time.
template <typename Real, typename T>
__device__ __forceinline__ void stage_rows(Real *dst, const T *src, int count, int w, int ld, int tid, int nthr) {
  constexpr int per = 16 / (int)sizeof(T);
  int done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int nv = count / per;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    for (int v = tid; v < nv; v += nthr) {
      const float4 c = __ldg(s4 + v);
      T vals[per];
      memcpy(vals, &c, sizeof(c));
      const int e = v * per;
      int r = e / w, col = e - r * w;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        dst[r * ld + col] = (Real)vals[q];
        if (++col == w) { col = 0; ++r; }
      }
    }
    done = nv * per;
  }
  for (int e = done + tid; e < count; e += nthr) {
    const int r = e / w, col = e - r * w;
    dst[r * ld + col] = (Real)__ldg(src + e);
  }
}

template <int NX, typename Real>
__device__ __forceinline__ void stage_blocks(Real *dst, const Real *src, int nblk, int ld, int tid, int T) {
  stage_rows(dst, src, nblk * NX * NX, NX, ld, tid, T);
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
  int ld, ldb;                                    // staged row strides
  int gld, gldb;                                  // row strides of gA and gPE, and of gB, in global memory
  bool gpad;                                      // gA, gB, gPE are the padded copies (16-byte aligned rows)
};

template <int NX, int OP, int RED, typename Real, bool CG = false, bool WARP = false>
__device__ void pcg_solve(const PcgArgs &a, const ProbDesc &d, Real *sm, typename Red<RED, Real>::T *slots) {
  using R = Red<RED, Real>;
  using AccT = typename R::T;
  constexpr int NXP = (NX + 3) & ~3;
  constexpr int NUC = (NX + 1) / 2;  // nu = ceil(nx / 2), the usual input count: unrolled B-row products
  const int p = d.id;  // output slot
  const int N = d.N, n = N + 1, nu = d.nu, R_ = n * NX, NUP = vec_stride(nu);
  const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x, T = WARP ? 32 : (int)blockDim.x;
  const int poly = a.poly;
  int K = pcg_max_resident(OP, N, NX, nu, a.smem_elems, poly > 0, CG);  // the host sized smem so that K >= 0
  if (K > a.max_resident) K = a.max_resident;
  if (K < 0) K = 0;
  if (N == 0) K = 1;  // a single knot is always staged, with its zero off-diagonal slot
  const int Ks = K < N ? K : N;
  const PcgLayout L = pcg_layout(OP, K, N, NX, nu, poly > 0, CG);
  Real *sp = sm + L.p, *sr = sm + L.r, *sw = sm + L.w, *sx = sm + L.x, *sv = sm + L.v, *se = sm + L.e;
  Real *su = sm + L.u, *ss = sm + L.s;
  Real *svu = sm + L.vu;  // v_u block rows, stride NUP
  // zero segments before block row 0 and after block row N of the vectors whose neighbour segments are read
  for (int e = tid; e < NXP; e += T) {
    sp[e - NXP] = Real(0); sp[n * NXP + e] = Real(0);
    sr[e - NXP] = Real(0); sr[n * NXP + e] = Real(0);
    sw[e - NXP] = Real(0); sw[n * NXP + e] = Real(0);
    if (poly > 0) { se[e - NXP] = Real(0); se[n * NXP + e] = Real(0); }
    if (CG) { su[e - NXP] = Real(0); su[n * NXP + e] = Real(0); }
    if (OP == kOpQp) sv[e - NXP] = Real(0);
  }
  if (OP == kOpQp)
    for (int e = tid; e < NUP; e += T) svu[e - NUP] = Real(0);
  // no off-diagonal preconditioner blocks (PE == nullptr): the preconditioner is block-diagonal
  const bool diag_only = a.PE == nullptr;
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
  // storage index of row (k, i) in the strided vectors
  auto vid = [&](int row, int &k, int &i) {
    k = row / NX;
    i = row - k * NX;
    return k * NXP + i;
  };

  // ---- views and staging ----
  Views<Real> V{};
  V.ld = pad_ld(NX);
  V.ldb = pad_ld(nu > 0 ? nu : 1);
  V.gld = NX; V.gldb = nu; V.gpad = false;
  V.gPD = reinterpret_cast<const Real *>(a.PD) + d.odiag;
  V.gPE = reinterpret_cast<const Real *>(a.PE) + d.ooff;
  {
    Real *spd = sm + L.pd, *spe = sm + L.pe;
    stage_blocks<NX>(spd, V.gPD, K, V.ld, tid, T);
    if (!diag_only) stage_blocks<NX>(spe, V.gPE, Ks, V.ld, tid, T);
    if (N == 0 && !diag_only)  // the zero off-diagonal slot of a single knot
      for (int e = tid; e < NX * V.ld; e += T) spe[e] = Real(0);
    V.sPD = spd; V.sPE = spe;
  }
  const float *gq = a.qd + d.oq, *gr = a.rd + d.orr;
  Real *siq = sm + L.iq, *sir = sm + L.ir;
  if constexpr (OP == kOpQp) {
    V.gA = a.A + d.oA;
    V.gB = a.B + d.oB;
    Real *s0 = sm + L.m0, *s1 = sm + L.m1;
    stage_rows(s0, V.gA, Ks * NX * NX, NX, V.ld, tid, T);
    if (nu > 0) stage_rows(s1, V.gB, Ks * NX * nu, nu, V.ldb, tid, T);
    if (N == 0) {  // the zero off-diagonal slot of a single knot
      for (int e = tid; e < NX * V.ld; e += T) s0[e] = Real(0);
      for (int e = tid; e < NX * V.ldb; e += T) s1[e] = Real(0);
    }
    for (int e = tid; e < R_; e += T) {
      const int k = e / NX, j = e - k * NX;
      siq[k * NXP + j] = Real(1) / (Real)gq[e];
    }
    for (int e = tid; e < N * nu; e += T) {
      const int k = e / nu, j = e - k * nu;
      sir[k * NUP + j] = Real(1) / (Real)gr[e];
    }
    V.sA = s0; V.sB = s1;
    // streamed block rows: the plan's padded copies of A, B and PE when it made them (rows of NXP, NUP
    // values, 16-byte aligned, so that row-wise reads take 128-bit loads), else the inputs themselves
    const int64_t po = (a.pad != nullptr && K < n) ? a.pad_off[p] : -1;
    if (po >= 0) {
      V.gpad = true;
      V.gld = NXP; V.gldb = NUP;
      V.gA = a.pad + po;
      V.gB = a.pad + po + pad_region((int64_t)N * NX, NX);
      V.gPE = reinterpret_cast<const Real *>(a.pad + po + pad_region((int64_t)N * NX, NX) +
                                             pad_region((int64_t)N * NX, nu));
    }
  } else {
    V.gD = a.D + d.odiag;
    V.gE = a.E + d.ooff;
    Real *s0 = sm + L.m0, *s1 = sm + L.m1;
    stage_rows(s0, V.gD, K * NX * NX, NX, V.ld, tid, T);
    stage_rows(s1, V.gE, Ks * NX * NX, NX, V.ld, tid, T);
    if (N == 0)  // the zero off-diagonal slot of a single knot
      for (int e = tid; e < NX * V.ld; e += T) s1[e] = Real(0);
    V.sD = s0; V.sE = s1;
  }

  // QP form, phase 1: sv = G^-1 C^T src (all threads), then a barrier.
  //   v_x(k)[j] = (-src_k[j] + sum_l A_k[l][j] src_{k+1}[l]) / q_k[j]
  //   v_u(k)[j] = (sum_l B_k[l][j] src_{k+1}[l]) / r_k[j]
  // Branch-free at k = N: the block index is clamped and src_{N+1} is the zero segment.
  auto apply_S_phase1 = [&](const Real *src) {
    if constexpr (OP == kOpQp) {
      const int nitems = R_ + N * nu;
      const float inv_nu = nu > 0 ? 1.0f / (float)nu : 0.0f;
      for (int it = tid; it < nitems; it += T) {
        if (it < R_) {
          const int k = it / NX, j = it - k * NX;
          const int kp = k < N ? k : (N > 0 ? N - 1 : 0);
          Seg<NX, Real> s;
          s.load(src + (k + 1) * NXP);
          const Real ax = k < K ? dot_seg<NX, true, Real>(V.sA + kp * NX * V.ld + j, V.ld, s.v)
                                : dot_seg<NX, false, Real>(V.gA + (int64_t)kp * NX * V.gld + j, V.gld, s.v);
          sv[k * NXP + j] = (-src[k * NXP + j] + ax) * siq[k * NXP + j];
        } else {
          const int t2 = it - R_;
          const int k = (int)(((float)t2 + 0.5f) * inv_nu);
          const int j = t2 - k * nu;
          Seg<NX, Real> s;
          s.load(src + (k + 1) * NXP);
          Real acc;
          if (k < K) acc = dot_seg<NX, true, Real>(V.sB + k * NX * V.ldb + j, V.ldb, s.v);
          else acc = dot_seg<NX, false, Real>(V.gB + (int64_t)k * NX * V.gldb + j, V.gldb, s.v);
          svu[k * NUP + j] = acc * sir[k * NUP + j];
        }
      }
      group_sync<WARP>();
    }
  };
  // Row (k, i) of S src (QP form: of C sv).
  //   w_k[i] = -v_x(k)[i] + A_{k-1}[i,:] v_x(k-1) + B_{k-1}[i,:] v_u(k-1)
  // Branch-free at k = 0: the block index is clamped and v_x(-1), v_u(-1) are zero segments.
  auto apply_S_row = [&](const Real *src, int k, int i) -> Real {
    if constexpr (OP == kOpQp) {
      const int km = k > 0 ? k - 1 : 0;
      Seg<NX, Real> s;
      s.load(sv + (k - 1) * NXP);
      const Real *vu = svu + (k - 1) * NUP;
      Real acc = -sv[k * NXP + i];
      Real ax, ab = Real(0);  // one accumulator, j in order: the sum order the parity runs were made with
      if (k < K) {
        ax = dot_seg<NX, true, Real>(V.sA + (km * NX + i) * V.ld, 1, s.v);
        const Real *Br = V.sB + (km * NX + i) * V.ldb;
        if (nu == NUC) {  // unrolled, v_u in registers (128-bit loads)
          Seg<NUC, Real> su_;
          su_.load(vu);
#pragma unroll
          for (int j = 0; j < NUC; ++j) ab = rfma(Br[j], su_.v[j], ab);
        } else {
          for (int j = 0; j < nu; ++j) ab = rfma(Br[j], vu[j], ab);
        }
      } else {
        const float *Br = V.gB + ((int64_t)km * NX + i) * V.gldb;
        if (V.gpad && nu == NUC) {  // padded rows: 128-bit loads; unrolled, v_u in registers
          ax = dot_row_g<NX, Real>(V.gA + ((int64_t)km * NX + i) * V.gld, s.v);
          Seg<NUC, Real> su_;
          su_.load(vu);
#pragma unroll
          for (int j4 = 0; j4 < NUC; j4 += 4) {
            const float4 bc = __ldg(reinterpret_cast<const float4 *>(Br + j4));
            const float *bq = reinterpret_cast<const float *>(&bc);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (j4 + t < NUC) ab = rfma((Real)bq[t], su_.v[j4 + t], ab);
          }
        } else if (V.gpad) {  // padded rows: 128-bit loads
          ax = dot_row_g<NX, Real>(V.gA + ((int64_t)km * NX + i) * V.gld, s.v);
          for (int j4 = 0; j4 < nu; j4 += 4) {
            const float4 bc = __ldg(reinterpret_cast<const float4 *>(Br + j4));
            const float *bq = reinterpret_cast<const float *>(&bc);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (j4 + t < nu) ab = rfma((Real)bq[t], vu[j4 + t], ab);
          }
        } else {
          ax = dot_seg<NX, false, Real>(V.gA + ((int64_t)km * NX + i) * NX, 1, s.v);
          for (int j = 0; j < nu; ++j) ab = rfma((Real)__ldg(Br + j), vu[j], ab);
        }
      }
      acc += ax;
      acc += ab;
      return acc;
    } else {
      return k < K ? bt_row<NX, true, Real>(V.sD, V.sE, V.ld, N, k, i, src)
                   : bt_row<NX, false, Real>(V.gD, V.gE, NX, N, k, i, src);
    }
  };
  auto apply_P_row = [&](const Real *src, int k, int i) -> Real {
    if (diag_only) {  // block-diagonal preconditioner: the diagonal block only (symmetric; read by column)
      Seg<NX, Real> s;
      s.load(src + k * NXP);
      return k < K ? dot_seg<NX, true, Real>(V.sPD + k * NX * V.ld + i, V.ld, s.v)
                   : dot_seg<NX, false, Real>(V.gPD + (int64_t)k * NX * NX + i, NX, s.v);
    }
    return k < K ? bt_row<NX, true, Real>(V.sPD, V.sPE, V.ld, N, k, i, src)
                 : bt_row_stream<NX, Real>(V.gPD, V.gPE, V.gld, V.gpad, N, k, i, src);
  };

  // dst = Phi_d^-1 sr (polynomial of degree d = poly, Horner correction form as in ``precondition``); ends
  // with a barrier.  The single-reduction variant's preconditioning step.
  auto precondition_into = [&](Real *dst) {
    for (int row = tid; row < R_; row += T) {
      int k, i;
      const int si = vid(row, k, i);
      dst[si] = apply_P_row(sr, k, i);
    }
    for (int t = 0; t < poly; ++t) {
      group_sync<WARP>();  // dst complete
      apply_S_phase1(dst);
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        se[si] = sr[si] - apply_S_row(dst, k, i);
      }
      group_sync<WARP>();  // e complete
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        dst[si] = dst[si] + apply_P_row(se, k, i);
      }
    }
    group_sync<WARP>();
  };

  // sw = z = Phi_d^-1 sr (polynomial of degree d = poly), and the block sums (r.z, r.r) into rz_, rr_.
  //   z = Phi^-1 r, then d times: e = r - S z, barrier, z += Phi^-1 e  (Eq. polynomial_precon:
  //   sum_{j<=d} (I - Phi^-1 S)^j Phi^-1 r in Horner form).  Ends with a barrier (the block sum).
  auto precondition = [&](Real &rz_, Real &rr_) {
    AccT s2[2] = {R::zero(), R::zero()};
    for (int row = tid; row < R_; row += T) {
      int k, i;
      const int si = vid(row, k, i);
      const Real z = apply_P_row(sr, k, i);
      const Real r = sr[si];
      sw[si] = z;
      if (poly == 0) s2[0] = R::fma(s2[0], r, z);
      s2[1] = R::fma(s2[1], r, r);
    }
    for (int t = 0; t < poly; ++t) {
      group_sync<WARP>();  // z complete
      apply_S_phase1(sw);
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        se[si] = sr[si] - apply_S_row(sw, k, i);
      }
      group_sync<WARP>();  // e complete
      const bool last = t + 1 == poly;
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        const Real z = sw[si] + apply_P_row(se, k, i);
        sw[si] = z;
        if (last) s2[0] = R::fma(s2[0], sr[si], z);
      }
    }
    group_sum<R, 2, WARP>(s2, slots + 64);
    rz_ = R::get(s2[0]);
    rr_ = R::get(s2[1]);
  };

  group_sync<WARP>();  // staged blocks and reciprocals visible

  // ---- r0 = gamma - S x0, z0 = Phi^-1 r0, p0 = z0 ----
  AccT g1[1] = {R::zero()};
  for (int row = tid; row < R_; row += T) {
    int k, i;
    const int si = vid(row, k, i);
    const Real g = (Real)gam[row];
    g1[0] = R::fma(g1[0], g, g);
    const Real x0 = a.warm ? lam_load(row) : Real(0);
    sp[si] = x0;
    sx[si] = x0;
  }
  group_sum<R, 1, WARP>(g1, slots);  // contains a barrier: sp complete
  const Real gg = R::get(g1[0]);
  const Real thresh = (Real)a.tol2 * gg;
  const int max_iter = a.max_iter > 0 ? a.max_iter : 10 * n * NX;
  if (gg == Real(0)) {
    for (int row = tid; row < R_; row += T) lam_store(row, Real(0));
    if (tid == 0) { a.iters[p] = 0; a.relres[p] = 0.0; a.status[p] = kOk; }
    group_sync<WARP>();
    return;
  }
  bool warm = a.warm != 0;
  if (warm) {
    apply_S_phase1(sp);
    for (int row = tid; row < R_; row += T) {
      int k, i;
      const int si = vid(row, k, i);
      sr[si] = (Real)gam[row] - apply_S_row(sp, k, i);
    }
  } else {
    for (int row = tid; row < R_; row += T) {
      int k, i;
      sr[vid(row, k, i)] = (Real)gam[row];
    }
  }
  group_sync<WARP>();
  if constexpr (CG) {
    // Single-reduction PCG (Chronopoulos & Gear 1989): the same iterates as the textbook algorithm, with
    // s = S p kept by recurrence, so that r.u, S u.u and r.r come from one block sum per iteration:
    //   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, barrier,
    //   u = Phi^-1 r, barrier, w = S u (QP form: phase 1, barrier, phase 2) with the three sums,
    //   beta = (r.u)new / (r.u), alpha = (r.u)new / ((S u.u) - beta (r.u)new / alpha)
    // since p.S p = S u.u - beta (r.u)new / alpha for the new p.  iters counts x updates, as textbook.
    Real ru = Real(0), del = Real(0), rr = Real(0);  // r.u, S u.u, r.r
    auto u_w_sums = [&]() {
      precondition_into(su);  // u = Phi_d^-1 r
      apply_S_phase1(su);
      AccT s3[3] = {R::zero(), R::zero(), R::zero()};
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        const Real w = apply_S_row(su, k, i);
        const Real u = su[si], r = sr[si];
        sw[si] = w;
        s3[0] = R::fma(s3[0], r, u);
        s3[1] = R::fma(s3[1], w, u);
        s3[2] = R::fma(s3[2], r, r);
      }
      group_sum<R, 3, WARP>(s3, slots);
      ru = R::get(s3[0]);
      del = R::get(s3[1]);
      rr = R::get(s3[2]);
    };
    for (int pass = 0; pass < 2; ++pass) {
      u_w_sums();
      if (pass == 0 && warm && a.warm == 2 && !(rr < gg)) {  // warm start no better than zero: restart
        for (int row = tid; row < R_; row += T) {
          int k, i;
          const int si = vid(row, k, i);
          sr[si] = (Real)gam[row];
          sx[si] = Real(0);
        }
        warm = false;
        group_sync<WARP>();
        continue;
      }
      break;
    }
    int it = 0, code = kOk;
    Real alpha = ru / del, beta = Real(0);
    if (!(del > Real(0)) || !isfinite(del)) code = isfinite(del) ? kBreakdown : kNonFinite;
    while (code == kOk) {
      if (!(rr > thresh)) {
        if (!isfinite(rr)) code = kNonFinite;
        break;
      }
      if (it >= max_iter) { code = kMaxIter; break; }
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        const Real pn = it == 0 ? su[si] : rfma(beta, sp[si], su[si]);
        const Real sn = it == 0 ? sw[si] : rfma(beta, ss[si], sw[si]);
        sp[si] = pn;
        ss[si] = sn;
        sx[si] = rfma(alpha, pn, sx[si]);
        sr[si] = rfma(-alpha, sn, sr[si]);
      }
      group_sync<WARP>();
      const Real ru_old = ru;
      u_w_sums();
      ++it;
      beta = ru / ru_old;
      const Real den = del - beta * ru / alpha;
      if (!(rr > thresh)) continue;  // converged: the next step is not taken
      if (!(den > Real(0)) || !isfinite(den)) { code = isfinite(den) ? kBreakdown : kNonFinite; break; }
      alpha = ru / den;
    }
    for (int row = tid; row < R_; row += T) {
      int k, i;
      lam_store(row, sx[vid(row, k, i)]);
    }
    if (tid == 0) {
      a.iters[p] = it;
      a.relres[p] = sqrt((double)rr / (double)gg);
      a.status[p] = code;
    }
    group_sync<WARP>();
    return;
  }
  Real rz, rr;
  for (int pass = 0; pass < 2; ++pass) {
    precondition(rz, rr);
    // warm start with fallback: restart from zero if lambda_0 is no better than zero
    if (pass == 0 && warm && a.warm == 2 && !(rr < gg)) {
      for (int row = tid; row < R_; row += T) {
        int k, i;
        const int si = vid(row, k, i);
        sr[si] = (Real)gam[row];
        sx[si] = Real(0);
      }
      warm = false;
      group_sync<WARP>();
      continue;
    }
    break;
  }
  for (int row = tid; row < R_; row += T) {
    int k, i;
    const int si = vid(row, k, i);
    sp[si] = sw[si];
  }
  group_sync<WARP>();

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
      int k, i;
      const int si = vid(row, k, i);
      const Real w = apply_S_row(sp, k, i);
      sw[si] = w;
      s1[0] = R::fma(s1[0], sp[si], w);
    }
    group_sum<R, 1, WARP>(s1, slots);
    const Real pw = R::get(s1[0]);
    if (!(pw > Real(0)) || !isfinite(pw)) { code = isfinite(pw) ? kBreakdown : kNonFinite; break; }
    const Real alpha = rz / pw;
    for (int row = tid; row < R_; row += T) {
      int k, i;
      const int si = vid(row, k, i);
      sx[si] = rfma(alpha, sp[si], sx[si]);
      sr[si] = rfma(-alpha, sw[si], sr[si]);
    }
    group_sync<WARP>();
    // z = Phi_d^-1 r, r.z, r.r
    Real rz_new;
    precondition(rz_new, rr);
    const Real beta = rz_new / rz;
    rz = rz_new;
    for (int row = tid; row < R_; row += T) {
      int k, i;
      const int si = vid(row, k, i);
      sp[si] = rfma(beta, sp[si], sw[si]);
    }
    group_sync<WARP>();
    ++it;
  }
  for (int row = tid; row < R_; row += T) {
    int k, i;
    lam_store(row, sx[vid(row, k, i)]);
  }
  if (tid == 0) {
    a.iters[p] = it;
    a.relres[p] = sqrt((double)rr / (double)gg);
    a.status[p] = code;
  }
  group_sync<WARP>();
}

// Persistent kernel: CTAs take problems from the work list, through an
// atomic counter when one is given (largest problems first), else by stride.
// GV: vectors in this CTA's slot of a global workspace (problems whose vectors do not fit in shared
// memory).  A compile-time choice, so that the other launches address their vectors as shared memory.
// WARP: every warp takes its own problems (one warp per problem, several per CTA); warp w of the CTA works in
// shared-memory slot w of a.smem_elems elements.
template <int NX, int OP, int RED, typename Real, bool GV, bool CG = false, bool WARP = false>
__global__ void __launch_bounds__(512) pcg_kernel(PcgArgs a) {
  extern __shared__ float4 smem4[];
  Real *sm;
  if constexpr (GV) sm = reinterpret_cast<Real *>(a.gscratch) + (int64_t)blockIdx.x * a.gstride;
  else sm = reinterpret_cast<Real *>(smem4);
  __shared__ __align__(16) typename Red<RED, Real>::T slots[4 * 32];
  __shared__ int s_next;
  int stride_i = 0;
  if constexpr (WARP) {
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Real *wsm = sm + (int64_t)wid * a.smem_elems;
    while (true) {
      int w;
      if (a.counter) {
        int t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(a.counter, 1);
        w = __shfl_sync(0xffffffffu, t, 0);
      } else {
        w = (blockIdx.x * nw + wid) + stride_i * gridDim.x * nw;
        ++stride_i;
      }
      if (w >= a.nwork) break;
      const ProbDesc d = a.ps.get(a.work ? a.work[w] : w);
      if (a.status[d.id] != kOk) continue;  // preconditioner failed for this problem
      pcg_solve<NX, OP, RED, Real, CG, true>(a, d, wsm, nullptr);
    }
  } else {
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
      pcg_solve<NX, OP, RED, Real, CG>(a, d, sm, slots);
    }
  }
}

// One compiled variant of the PCG kernel: its launch and its occupancy (CTAs per SM for a block size and
// dynamic shared memory, registers included).  The shared-memory attribute is set once per device.
// WARP launches split the dynamic shared memory into one slot per warp (a multiple of 16 bytes each).
template <int NX, int OP, int RED, typename Real, bool GV, bool CG, bool WARP = false>
struct PcgVariant {
  static cudaError_t prepare() {
    static std::atomic<uint64_t> attr_done{0};
    return smem_attr_once(attr_done, pcg_kernel<NX, OP, RED, Real, GV, CG, WARP>, pcg_max_smem_bytes());
  }
  static cudaError_t launch(const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    PcgArgs b = a;
    if constexpr (WARP) {
      if (block % 32 != 0) return cudaErrorInvalidValue;
      b.smem_elems = (int64_t)((smem / (size_t)(block / 32)) & ~(size_t)15) / (int64_t)sizeof(Real);
    } else {
      b.smem_elems = (int64_t)(smem / sizeof(Real));
    }
    pcg_kernel<NX, OP, RED, Real, GV, CG, WARP><<<grid, block, smem, st>>>(b);
    return cudaGetLastError();
  }
  static cudaError_t occupancy(int block, size_t smem, int *ctas) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, pcg_kernel<NX, OP, RED, Real, GV, CG, WARP>, block,
                                                         smem);
  }
};

// The variant of one nx for an operator form, reduction mode and precision: FP32 with three reduction modes
// for both operator forms, and the FP64 path (QP form, FP64 reductions); vectors in a global workspace (gv)
// for the QP form only; single-reduction PCG (cg) for the QP form with FP32 arithmetic and double-float sums.
// f(PcgVariant<...>{}) is called on it; cudaErrorInvalidValue when no variant exists.
// warp: one problem per warp, for the QP form with textbook PCG: FP32 with double-float sums, and the FP64
// path.
template <int NX, typename F>
cudaError_t with_pcg_variant(int op, int red, bool f64, bool gv, bool cg, bool warp, F &&f) {
  if (warp) {
    if (op != kOpQp || gv || (cg && !f64)) return cudaErrorInvalidValue;
    if (f64) return f(PcgVariant<NX, kOpQp, kRedF64, double, false, false, true>{});
    if (red == kRedDf) return f(PcgVariant<NX, kOpQp, kRedDf, float, false, false, true>{});
    return cudaErrorInvalidValue;
  }
  if (cg && op == kOpQp && !f64) {  // single-reduction PCG (the FP64 and block-form launches stay textbook)
    if (red != kRedDf) return cudaErrorInvalidValue;
    if (gv) return f(PcgVariant<NX, kOpQp, kRedDf, float, true, true>{});
    return f(PcgVariant<NX, kOpQp, kRedDf, float, false, true>{});
  }
  if (gv) {
    if (op != kOpQp) return cudaErrorInvalidValue;
    if (f64) return f(PcgVariant<NX, kOpQp, kRedF64, double, true, false>{});
    if (red == kRedDf) return f(PcgVariant<NX, kOpQp, kRedDf, float, true, false>{});
    if (red == kRedF32) return f(PcgVariant<NX, kOpQp, kRedF32, float, true, false>{});
    if (red == kRedF64) return f(PcgVariant<NX, kOpQp, kRedF64, float, true, false>{});
    return cudaErrorInvalidValue;
  }
  if (f64) {
    if (op != kOpQp) return cudaErrorInvalidValue;
    return f(PcgVariant<NX, kOpQp, kRedF64, double, false, false>{});
  }
#define SSPCG_PCG_CASE(OPV, REDV) \
  if (op == OPV && red == REDV) return f(PcgVariant<NX, OPV, REDV, float, false, false>{});
  SSPCG_PCG_CASE(kOpQp, kRedDf)
  SSPCG_PCG_CASE(kOpQp, kRedF32)
  SSPCG_PCG_CASE(kOpQp, kRedF64)
  SSPCG_PCG_CASE(kOpBlock, kRedDf)
  SSPCG_PCG_CASE(kOpBlock, kRedF32)
  SSPCG_PCG_CASE(kOpBlock, kRedF64)
#undef SSPCG_PCG_CASE
  return cudaErrorInvalidValue;
}

template <int NX>
cudaError_t launch_pcg_for_nx(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem,
                              cudaStream_t st) {
  return with_pcg_variant<NX>(op, red, f64, a.gscratch != nullptr, a.cg != 0, a.warp != 0,
                              [&](auto v) { return decltype(v)::launch(a, grid, block, smem, st); });
}

template <int NX>
cudaError_t occupancy_pcg_for_nx(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem,
                                 int *ctas) {
  return with_pcg_variant<NX>(op, red, f64, gv, cg, warp,
                              [&](auto v) { return decltype(v)::occupancy(block, smem, ctas); });
}

}  // namespace sspcg

#define SSPCG_INSTANTIATE_PCG(NXV)                                                                           \
  namespace sspcg {                                                                                          \
  cudaError_t launch_pcg_nx##NXV(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, \
                                 cudaStream_t st) {                                                          \
    return launch_pcg_for_nx<NXV>(op, red, f64, a, grid, block, smem, st);                                    \
  }                                                                                                          \
  cudaError_t occupancy_pcg_nx##NXV(int op, int red, bool f64, bool gv, bool cg, bool warp, int block,        \
                                    size_t smem, int *ctas) {                                                \
    return occupancy_pcg_for_nx<NXV>(op, red, f64, gv, cg, warp, block, smem, ctas);                          \
  }                                                                                                          \
  }
