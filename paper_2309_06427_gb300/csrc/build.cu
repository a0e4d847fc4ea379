// Schur-block build (Sec. II-A) and preconditioner assembly (Eq. stair_inv,
// Sec. III, Sec. IV, Eq. jacobi).  One warp per knot; the batch is a flat
// list of knots whose (problem, block row) pairs the plan tabulates.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace sspcg {

constexpr int kBuildWarps = 8;  // warps per CTA of the build kernels

// ---------------------------------------------------------------------------
// K1: D_k, E_k from (A, B, diag Q, diag R).
//   D_0 = Q_0^-1
//   D_k = A_{k-1} Q_{k-1}^-1 A_{k-1}^T + B_{k-1} R_{k-1}^-1 B_{k-1}^T + Q_k^-1   (= -theta_{k-1})
//   E[k-1] = S(k, k-1) = -A_{k-1} Q_{k-1}^-1                                   (= -phi_{k-1})
// Real = float (FP32 arithmetic) or double (the FP64 path); only the upper
// triangle of D_k is summed and mirrored, so D_k is exactly symmetric.
// Shared memory per warp: AQ, A, BR, B (mx*mx each, mx = largest nx, nu of the launch), 1/q_k (mx).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kBuildWarps * 32) schur_build_kernel(ProbSet ps, const int2 *refs,
                                                                      int64_t total_knots, const float *__restrict__ A,
                                                                      const float *__restrict__ B,
                                                                      const float *__restrict__ qd,
                                                                      const float *__restrict__ rd, Real *D, Real *E,
                                                                      int mx) {
  extern __shared__ float4 smem_raw[];
  Real *smem = reinterpret_cast<Real *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per_warp = 4 * mx * mx + mx;  // mx: largest nx (and nu) of the launch
  Real *sAQ = smem + wid * per_warp;
  Real *sA = sAQ + mx * mx;
  Real *sBR = sA + mx * mx;
  Real *sB = sBR + mx * mx;
  Real *sIq = sB + mx * mx;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_knots; g += (int64_t)gridDim.x * kBuildWarps) {
    const int2 ref = refs ? refs[g] : make_int2(0, (int)g);  // (problem, block row)
    const ProbDesc d = ps.get(ref.x);
    const int k = ref.y;
    const int nx = d.nx, nu = d.nu, nn = nx * nx;
    Real *Dk = D + d.odiag + (int64_t)k * nn;
    if (k == 0) {
      const float *q0 = qd + d.oq;
      for (int e = lane; e < nn; e += 32) {
        const int i = e / nx, j = e - i * nx;
        Dk[e] = (i == j) ? Real(1) / (Real)q0[i] : Real(0);
      }
      continue;
    }
    const float *Ak = A + d.oA + (int64_t)(k - 1) * nn;
    const float *Bk = B + d.oB + (int64_t)(k - 1) * nx * nu;
    const float *qp = qd + d.oq + (int64_t)(k - 1) * nx;
    const float *qk = qd + d.oq + (int64_t)k * nx;
    const float *rp = rd + d.orr + (int64_t)(k - 1) * nu;
    Real *Ek = E + d.ooff + (int64_t)(k - 1) * nn;
#pragma unroll 4
    for (int e = lane; e < nn; e += 32) {
      const int l = e % nx;
      const Real a = (Real)Ak[e];
      const Real aq = a / (Real)qp[l];
      sA[e] = a;
      sAQ[e] = aq;
      Ek[e] = -aq;
    }
    for (int e = lane; e < nx * nu; e += 32) {
      const int m = e % nu;
      const Real b = (Real)Bk[e];
      sB[e] = b;
      sBR[e] = b / (Real)rp[m];
    }
    for (int i = lane; i < nx; i += 32) sIq[i] = Real(1) / (Real)qk[i];
    __syncwarp();
    // upper triangle in tiles of four entries of one row, (i, j0..j0+3) with j0 = i + 4 t: each lane keeps four
    // accumulators and loads the row-i factor once per term; every entry sums its terms in the same order
    // as a one-entry loop would (l = 0..nx-1, then m = 0..nu-1)
    const int ntiles = (nx * (nx + 1) / 2 + 3 * nx) / 4 + nx;  // an upper bound; tiles past the end are skipped
    for (int tl = lane; tl < ntiles; tl += 32) {
      int i = 0, rem = tl;
      while (i < nx && rem >= (nx - i + 3) / 4) rem -= (nx - i + 3) / 4, ++i;
      if (i >= nx) break;
      const int j0 = i + 4 * rem;
      int jj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) jj[q] = min(j0 + q, nx - 1);
      Real s[4] = {Real(0), Real(0), Real(0), Real(0)};
      for (int l = 0; l < nx; ++l) {
        const Real a = sAQ[i * nx + l];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = fma(a, sA[jj[q] * nx + l], s[q]);
      }
      for (int m = 0; m < nu; ++m) {
        const Real b = sBR[i * nu + m];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = fma(b, sB[jj[q] * nu + m], s[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        if (j >= nx) break;
        Real v = s[q];
        if (i == j) v += sIq[i];
        Dk[i * nx + j] = v;
        Dk[j * nx + i] = v;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K1 with full SPD cost blocks (Sec. II-A, Q_k^-1 and R_k^-1 as matrices), from
// their inverses Qi (laid out like D) and Ri (R_{k-1}^-1 at roff[p] + (k-1) nu^2):
//   D_0 = Q_0^-1
//   D_k = (A_{k-1} Q_{k-1}^-1) A_{k-1}^T + (B_{k-1} R_{k-1}^-1) B_{k-1}^T + Q_k^-1
//   E[k-1] = -A_{k-1} Q_{k-1}^-1
// FP32; the upper triangle of D_k is summed and mirrored (Q_k^-1 is exactly
// symmetric), so D_k is exactly symmetric.  One warp per knot.
// Shared memory per warp: A, Q^-1, A Q^-1, B, R^-1, B R^-1 (mx*mx each).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBuildWarps * 32) schur_full_kernel(ProbSet ps, const int2 *refs,
                                                                     int64_t total_knots, const int64_t *roff,
                                                                     const float *__restrict__ A,
                                                                     const float *__restrict__ B,
                                                                     const float *__restrict__ Qi,
                                                                     const float *__restrict__ Ri, float *D, float *E,
                                                                     int mx) {
  extern __shared__ float4 smem_raw[];
  float *smem = reinterpret_cast<float *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int mm = mx * mx;
  float *sA = smem + wid * 6 * mm, *sQ = sA + mm, *sAQ = sQ + mm, *sB = sAQ + mm, *sR = sB + mm, *sBR = sR + mm;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_knots; g += (int64_t)gridDim.x * kBuildWarps) {
    const int2 ref = refs ? refs[g] : make_int2(0, (int)g);  // (problem, block row)
    const ProbDesc d = ps.get(ref.x);
    const int k = ref.y;
    const int nx = d.nx, nu = d.nu, nn = nx * nx;
    float *Dk = D + d.odiag + (int64_t)k * nn;
    const float *Qk = Qi + d.odiag + (int64_t)k * nn;
    if (k == 0) {
      for (int e = lane; e < nn; e += 32) Dk[e] = Qk[e];
      continue;
    }
    const float *Ak = A + d.oA + (int64_t)(k - 1) * nn;
    const float *Bk = B + d.oB + (int64_t)(k - 1) * nx * nu;
    const float *Qp = Qi + d.odiag + (int64_t)(k - 1) * nn;
    const float *Rp = Ri + (roff ? roff[ref.x] : 0) + (int64_t)(k - 1) * nu * nu;
    float *Ek = E + d.ooff + (int64_t)(k - 1) * nn;
    for (int e = lane; e < nn; e += 32) {
      sA[e] = Ak[e];
      sQ[e] = Qp[e];
    }
    for (int e = lane; e < nx * nu; e += 32) sB[e] = Bk[e];
    for (int e = lane; e < nu * nu; e += 32) sR[e] = Rp[e];
    __syncwarp();
    for (int e = lane; e < nn; e += 32) {
      const int i = e / nx, j = e - i * nx;
      float s = 0.0f;
      for (int l = 0; l < nx; ++l) s = fmaf(sA[i * nx + l], sQ[l * nx + j], s);
      sAQ[e] = s;
      Ek[e] = -s;
    }
    for (int e = lane; e < nx * nu; e += 32) {
      const int i = e / nu, j = e - i * nu;
      float s = 0.0f;
      for (int m = 0; m < nu; ++m) s = fmaf(sB[i * nu + m], sR[m * nu + j], s);
      sBR[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < nn; e += 32) {
      const int i = e / nx, j = e - i * nx;
      if (i > j) continue;
      float s = 0.0f;
      for (int l = 0; l < nx; ++l) s = fmaf(sAQ[i * nx + l], sA[j * nx + l], s);
      for (int m = 0; m < nu; ++m) s = fmaf(sBR[i * nu + m], sB[j * nu + m], s);
      s += Qk[i * nx + j];
      Dk[i * nx + j] = s;
      Dk[j * nx + i] = s;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K2a: PD_k = D_k^-1 by LDL^T in FP64 (FP64 output) or double-float (FP32
// output: about 48 bits on the FP32 units; GB300 issues FP64 at about 1/64 of
// the FP32 rate), G lanes per knot (all knots of a launch have the same nx).
// In shared memory per knot: the packed lower triangle of D_k (8-byte entries,
// odd stride for conflict-free accesses).
//   LDL^T, right-looking:                               nx^3/6 FMA
//   L^-1 in place (unit lower), row by row:             nx^3/6 FMA
//   D^-1(i,j) = sum_{t>=i} W(t,i) (1/d_t) W(t,j), i >= j:  nx^3/6 FMA
// Reciprocals: FP32 reciprocal refined by Newton steps (two in FP64, one in
// double-float).  Jacobi: PD_k = diag(1 / D_k(i,i)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_f64(double x) {
  double y = (double)(1.0f / (float)x);
  y = y * fma(-x, y, 2.0);
  y = y * fma(-x, y, 2.0);
  return y;
}

// Per-thread storage: the packed lower triangle, row i at offset i(i+1)/2;
// the per-thread stride is odd (8-byte words) so that a warp's accesses to
// the same entry fall in distinct banks.
__host__ __device__ __forceinline__ int inv_stride(int nx) { return (nx * (nx + 1) / 2) | 1; }
__device__ __forceinline__ int tri(int i, int c) { return i * (i + 1) / 2 + c; }

// D_k^-1 by FP64 LDL^T and D^-1 = V^T V with V = diag(1/d)^(1/2) L^-1, G lanes per knot: the G lanes of a group share the
// knot's packed triangle in shared memory and split the rows (LDL^T update,
// D^-1 entries) or the columns (the triangular inverse) between them, so the
// same shared memory holds G times more warps than one knot per thread.  All
// knots of a launch have the same nx, so the lanes of a warp run the same
// loops and synchronise with __syncwarp over the warp's active lanes.  Every
// entry is computed with the same operations in the same order as one lane
// would, so the result does not depend on G.
// Arithmetic of the inversion: FP64 for the FP64 path (FP64 output), double-float for FP32 output (about 48
// bits on the FP32 units, which run at about 60x the FP64 rate; the output is rounded to FP32 once).  Both
// run the same operations in the same order.
template <typename T> struct InvArith;
template <> struct InvArith<double> {
  using T = double;
  static __device__ __forceinline__ T from(double v) { return v; }
  static __device__ __forceinline__ T fnma(T a, T b, T c) { return fma(-a, b, c); }  // c - a b
  static __device__ __forceinline__ T fma3(T a, T b, T c) { return fma(a, b, c); }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T rcp(T a) { return rcp_f64(a); }
  static __device__ __forceinline__ T sqrt_(T a) { return sqrt(a); }
  static __device__ __forceinline__ bool pos_finite(T a) { return a > 0.0 && isfinite(a); }
  template <typename Real> static __device__ __forceinline__ Real out(T a) { return (Real)a; }
};
template <> struct InvArith<df> {
  using T = df;
  static __device__ __forceinline__ T from(float v) { return {v, 0.0f}; }
  static __device__ __forceinline__ T fnma(T a, T b, T c) { return df_fma3(df_neg(a), b, c); }
  static __device__ __forceinline__ T fma3(T a, T b, T c) { return df_fma3(a, b, c); }
  static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
  static __device__ __forceinline__ T rcp(T a) { return df_rcp(a); }
  static __device__ __forceinline__ T sqrt_(T a) { return df_sqrt(a); }
  static __device__ __forceinline__ bool pos_finite(T a) { return a.hi > 0.0f && isfinite(a.hi); }
  template <typename Real> static __device__ __forceinline__ Real out(T a) { return (Real)__fadd_rn(a.hi, a.lo); }
};

template <typename Real, int G>
__global__ void __launch_bounds__(512, 1) precond_inv_kernel(ProbSet ps, const int2 *refs, int64_t total_knots, int nx,
                                                          int kind, const Real *__restrict__ D, Real *PD,
                                                          int32_t *status) {
  using A = InvArith<typename std::conditional<sizeof(Real) == sizeof(float), df, double>::type>;
  using T = typename A::T;
  static_assert(sizeof(T) == sizeof(double), "8-byte entries: the shared-memory layout is the same for both");
  extern __shared__ double dsm[];
  const int lg = threadIdx.x % G, grp = threadIdx.x / G;
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x / G) + grp;
  const bool active = g < total_knots;
  const unsigned mask = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const int2 ref = refs ? refs[g] : make_int2(0, (int)g);  // (problem, block row)
  const ProbDesc d = ps.get(ref.x);
  const int k = ref.y;
  const int nn = nx * nx;
  const Real *Dk = D + d.odiag + (int64_t)k * nn;
  Real *PDk = PD + d.odiag + (int64_t)k * nn;
  if (kind == 3) {  // Jacobi: reciprocal diagonal
    bool bad = false;
    for (int e = lg; e < nn; e += G) PDk[e] = Real(0);
    __syncwarp(mask);
    for (int i = lg; i < nx; i += G) {
      const Real s = Dk[i * nx + i];
      bad |= !(s > Real(0)) || !isfinite(s);
      PDk[i * nx + i] = Real(1) / s;
    }
    if (bad) status[d.id] = kNotSpd;
    return;
  }
  T *M = reinterpret_cast<T *>(dsm) + (int64_t)grp * (inv_stride(nx) + nx);
  T *tmp = M + inv_stride(nx);
  for (int i = 0; i < nx; ++i)
    for (int c = lg; c <= i; c += G) M[tri(i, c)] = A::from(Dk[i * nx + c]);
  __syncwarp(mask);
  // LDL^T: after step j, M(j,j) = 1/d_j and M(i,j) = L(i,j) for i > j.  Rows i > j are split cyclically.
  bool bad = false;
  for (int j = 0; j < nx; ++j) {
    const T djj = M[tri(j, j)];
    bad |= !A::pos_finite(djj);
    const T inv = A::rcp(djj);
    for (int i = j + 1 + lg; i < nx; i += G) {
      T *Mi = M + tri(i, 0);
      const T lij = A::mul(Mi[j], inv);
#pragma unroll 4
      for (int c = j + 1; c <= i; ++c) Mi[c] = A::fnma(lij, M[tri(c, j)], Mi[c]);
    }
    __syncwarp(mask);  // column j no longer read
    for (int i = j + 1 + lg; i < nx; i += G) M[tri(i, j)] = A::mul(M[tri(i, j)], inv);
    if (lg == 0) M[tri(j, j)] = inv;
    __syncwarp(mask);
  }
  // W = L^-1 (unit lower) in place, row by row; the columns of a row are split cyclically.
  //   W(i,j) = -(L(i,j) + sum_{j<t<i} L(i,t) W(t,j))
  for (int i = 1; i < nx; ++i) {
    const T *Mi = M + tri(i, 0);
    for (int j = lg; j < i; j += G) {
      T s0 = Mi[j], s1 = A::from(0.0f);  // two chains
      int t = j + 1;
      for (; t + 1 < i; t += 2) {
        s0 = A::fma3(Mi[t], M[tri(t, j)], s0);
        s1 = A::fma3(Mi[t + 1], M[tri(t + 1, j)], s1);
      }
      if (t < i) s0 = A::fma3(Mi[t], M[tri(t, j)], s0);
      tmp[j] = A::neg(A::add(s0, s1));
    }
    __syncwarp(mask);  // row i's L entries no longer read
    for (int j = lg; j < i; j += G) M[tri(i, j)] = tmp[j];
    __syncwarp(mask);
  }
  // FP32 output: V = diag(1/d)^(1/2) W (row t of W scaled by sqrt(1/d_t); V(t,t) = sqrt(1/d_t)), so that
  // D^-1 = W^T diag(1/d) W = V^T V costs one FMA per term.  Rows split cyclically.  FP64 output keeps
  // W^T diag(1/d) W term by term (two operations per term, the rounding the FP64 path is checked with).
  constexpr bool kVtV = sizeof(Real) == sizeof(float);
  if (kVtV && !bad) {
    for (int t = lg; t < nx; t += G) {
      T *Mt = M + tri(t, 0);
      const T sc = A::sqrt_(Mt[t]);
      for (int c = 0; c < t; ++c) Mt[c] = A::mul(Mt[c], sc);
      Mt[t] = sc;
    }
  }
  __syncwarp(mask);  // the last synchronisation: groups may leave from here on
  if (bad) {
    if (lg == 0) status[d.id] = kNotSpd;
    for (int e = lg; e < nn; e += G) PDk[e] = Real(0);
    return;
  }
  // D^-1(i,j): lower-triangle entries split cyclically, mirrored.
  const int npairs = nx * (nx + 1) / 2;
  for (int e = lg; e < npairs; e += G) {
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (tri(i + 1, 0) <= e) ++i;
    while (tri(i, 0) > e) --i;
    const int j = e - tri(i, 0);
    T s0, s1 = A::from(0.0f);  // two chains
    int t = i + 1;
    if constexpr (kVtV) {
      s0 = A::mul(M[tri(i, i)], M[tri(i, j)]);
      for (; t + 1 < nx; t += 2) {
        const T *Mt = M + tri(t, 0), *Mu = M + tri(t + 1, 0);
        s0 = A::fma3(Mt[i], Mt[j], s0);
        s1 = A::fma3(Mu[i], Mu[j], s1);
      }
      if (t < nx) {
        const T *Mt = M + tri(t, 0);
        s0 = A::fma3(Mt[i], Mt[j], s0);
      }
    } else {
      s0 = A::mul(M[tri(i, i)], i == j ? A::from(1.0f) : M[tri(i, j)]);
      for (; t + 1 < nx; t += 2) {
        const T *Mt = M + tri(t, 0), *Mu = M + tri(t + 1, 0);
        s0 = A::fma3(A::mul(Mt[i], Mt[t]), Mt[j], s0);
        s1 = A::fma3(A::mul(Mu[i], Mu[t + 1]), Mu[j], s1);
      }
      if (t < nx) {
        const T *Mt = M + tri(t, 0);
        s0 = A::fma3(A::mul(Mt[i], Mt[t]), Mt[j], s0);
      }
    }
    const Real f = A::template out<Real>(A::add(s0, s1));
    PDk[i * nx + j] = f;
    PDk[j * nx + i] = f;
  }
}

// ---------------------------------------------------------------------------
// K2b: PE[k-1] = -c * PD_k E[k-1] PD_{k-1}, c = 1 (symmetric stair) or 1/2
// (additive stair), in Real.  One warp per off-diagonal block.
// Shared memory per warp: PD_k, E, PD_{k-1}, T = PD_k E (4 * mx * mx elements).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kBuildWarps * 32) precond_off_kernel(ProbSet ps, const int2 *refs,
                                                                      int64_t total_off, Real c,
                                                                      const Real *__restrict__ E,
                                                                      const Real *__restrict__ PD, Real *PE, int mx) {
  extern __shared__ float4 smem_raw[];
  Real *smem = reinterpret_cast<Real *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per_warp = 4 * mx * mx;  // mx: largest nx of the launch
  Real *sP1 = smem + wid * per_warp;
  Real *sE = sP1 + mx * mx;
  Real *sP0 = sE + mx * mx;
  Real *sT = sP0 + mx * mx;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_off; g += (int64_t)gridDim.x * kBuildWarps) {
    const int2 ref = refs ? refs[g] : make_int2(0, (int)g + 1);  // (problem, block row k >= 1)
    const ProbDesc d = ps.get(ref.x);
    const int k = ref.y;
    const int nx = d.nx, nn = nx * nx;
    const Real *P1 = PD + d.odiag + (int64_t)k * nn;
    const Real *P0 = PD + d.odiag + (int64_t)(k - 1) * nn;
    const Real *Ek = E + d.ooff + (int64_t)(k - 1) * nn;
    Real *PEk = PE + d.ooff + (int64_t)(k - 1) * nn;
#pragma unroll 4
    for (int e = lane; e < nn; e += 32) {
      sP1[e] = P1[e];
      sE[e] = Ek[e];
      sP0[e] = P0[e];
    }
    __syncwarp();
    // both products in tiles of four entries of one row, (i, 4 t .. 4 t + 3): four accumulators per lane, the
    // row factor loaded once per term; each entry sums t = 0..nx-1 in order, as a one-entry loop would
    const int cw = (nx + 3) / 4, ntl = nx * cw;
    for (int tl = lane; tl < ntl; tl += 32) {
      const int i = tl / cw, j0 = 4 * (tl - i * cw);
      int jj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) jj[q] = min(j0 + q, nx - 1);
      Real s[4] = {Real(0), Real(0), Real(0), Real(0)};
      for (int t = 0; t < nx; ++t) {
        const Real a = sP1[i * nx + t];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = fma(a, sE[t * nx + jj[q]], s[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j0 + q < nx) sT[i * nx + j0 + q] = s[q];
    }
    __syncwarp();
    for (int tl = lane; tl < ntl; tl += 32) {
      const int i = tl / cw, j0 = 4 * (tl - i * cw);
      int jj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) jj[q] = min(j0 + q, nx - 1);
      Real s[4] = {Real(0), Real(0), Real(0), Real(0)};
      for (int t = 0; t < nx; ++t) {
        const Real a = sT[i * nx + t];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = fma(a, sP0[t * nx + jj[q]], s[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        if (j >= nx) break;
        const Real v = -c * s[q];
        PEk[i * nx + j] = v;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
static int build_grid(int64_t items, int sms) {
  (void)sms;
  const int64_t need = cdiv(items, kBuildWarps);  // one warp per item
  const int64_t cap = 1 << 30;
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

template <typename Real>
cudaError_t launch_schur_build(const ProbSet &ps, const int2 *refs, int64_t total_knots, const float *A,
                               const float *B, const float *qd, const float *rd, Real *D, Real *E,
                               cudaStream_t st, int sms, int mx) {
  if (total_knots == 0) return cudaSuccess;
  const size_t smem = sizeof(Real) * kBuildWarps * (4 * mx * mx + mx);
  static std::atomic<uint64_t> attr_done{0};
  const size_t most = sizeof(Real) * kBuildWarps * (4 * kMaxNx * kMaxNx + kMaxNx);
  cudaError_t e = smem_attr_once(attr_done, schur_build_kernel<Real>, (int)most);
  if (e != cudaSuccess) return e;
  schur_build_kernel<Real><<<build_grid(total_knots, sms), kBuildWarps * 32, smem, st>>>(ps, refs, total_knots,
                                                                                          A, B, qd, rd, D, E, mx);
  return cudaGetLastError();
}

cudaError_t launch_schur_full(const ProbSet &ps, const int2 *refs, int64_t total_knots, const int64_t *roff,
                              const float *A, const float *B, const float *Qi, const float *Ri, float *D, float *E,
                              cudaStream_t st, int mx) {
  if (total_knots == 0) return cudaSuccess;
  const size_t smem = sizeof(float) * kBuildWarps * 6 * mx * mx;
  static std::atomic<uint64_t> attr_done{0};
  const size_t most = sizeof(float) * kBuildWarps * 6 * kMaxNx * kMaxNx;
  cudaError_t e = smem_attr_once(attr_done, schur_full_kernel, (int)most);
  if (e != cudaSuccess) return e;
  schur_full_kernel<<<build_grid(total_knots, 0), kBuildWarps * 32, smem, st>>>(ps, refs, total_knots, roff, A, B,
                                                                                 Qi, Ri, D, E, mx);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_precond_inv(const ProbSet &ps, const int2 *refs, int64_t total_knots, int nx, int kind,
                               const Real *D, Real *PD, int32_t *status, cudaStream_t st) {
  if (total_knots == 0) return cudaSuccess;
  static std::atomic<uint64_t> attr4{0}, attr8{0};
  cudaError_t e = smem_attr_once(attr4, precond_inv_kernel<Real, 4>, 210 * 1024);
  if (e == cudaSuccess) e = smem_attr_once(attr8, precond_inv_kernel<Real, 8>, 210 * 1024);
  if (e != cudaSuccess) return e;
  // lanes per knot: 8 for the larger blocks, 4 otherwise; knots per CTA limited by 112 KB of shared memory, so
  // that two CTAs fit on an SM (about 28 warps per SM for nx = 21 instead of 16)
  const int G = nx >= 16 ? 8 : 4;
  const int per_knot = (inv_stride(nx) + nx) * (int)sizeof(double);
  int knots = (int)std::min<int64_t>(512 / G, (112 * 1024) / per_knot);
  knots = std::max(32 / G, knots / (32 / G) * (32 / G));  // whole warps
  const int threads = knots * G;
  const size_t smem = kind == 3 ? 0 : (size_t)knots * per_knot;
  const unsigned grid = (unsigned)cdiv(total_knots, knots);
  if (G == 8)
    precond_inv_kernel<Real, 8><<<grid, threads, smem, st>>>(ps, refs, total_knots, nx, kind, D, PD, status);
  else
    precond_inv_kernel<Real, 4><<<grid, threads, smem, st>>>(ps, refs, total_knots, nx, kind, D, PD, status);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_precond_off(const ProbSet &ps, const int2 *refs, int64_t total_off, int kind,
                               const Real *E, const Real *PD, Real *PE, cudaStream_t st, int sms, int64_t off_elems,
                               int mx) {
  if (total_off == 0) return cudaSuccess;
  if (kind == 2 || kind == 3) {  // block-Jacobi, Jacobi: no off-diagonal blocks
    return cudaMemsetAsync(PE, 0, sizeof(Real) * off_elems, st);
  }
  const size_t smem_o = sizeof(Real) * kBuildWarps * (4 * mx * mx);
  static std::atomic<uint64_t> attr_done{0};
  const size_t most = sizeof(Real) * kBuildWarps * (4 * kMaxNx * kMaxNx);
  cudaError_t e = smem_attr_once(attr_done, precond_off_kernel<Real>, (int)most);
  if (e != cudaSuccess) return e;
  const Real c = (kind == 0) ? Real(1) : Real(0.5);
  precond_off_kernel<Real><<<build_grid(total_off, sms), kBuildWarps * 32, smem_o, st>>>(ps, refs, total_off, c,
                                                                                          E, PD, PE, mx);
  return cudaGetLastError();
}

template cudaError_t launch_schur_build<float>(const ProbSet &, const int2 *, int64_t, const float *, const float *,
                                               const float *, const float *, float *, float *, cudaStream_t, int,
                                               int);
template cudaError_t launch_schur_build<double>(const ProbSet &, const int2 *, int64_t, const float *,
                                                const float *, const float *, const float *, double *, double *,
                                                cudaStream_t, int, int);
template cudaError_t launch_precond_inv<float>(const ProbSet &, const int2 *, int64_t, int, int, const float *,
                                               float *, int32_t *, cudaStream_t);
template cudaError_t launch_precond_inv<double>(const ProbSet &, const int2 *, int64_t, int, int, const double *,
                                                double *, int32_t *, cudaStream_t);
template cudaError_t launch_precond_off<float>(const ProbSet &, const int2 *, int64_t, int, const float *,
                                               const float *, float *, cudaStream_t, int, int64_t, int);
template cudaError_t launch_precond_off<double>(const ProbSet &, const int2 *, int64_t, int, const double *,
                                                const double *, double *, cudaStream_t, int, int64_t, int);

}  // namespace sspcg
