// Shared device-side definitions of the sspcg CUDA library (sm_103a).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace sspcg {

constexpr int kMaxNx = 28;

// Per-problem solve outcome codes (same values as the SSPCG_SOLVE_* enum of sspcg.h).
enum SolveCode : int { kOk = 0, kMaxIter = 1, kBreakdown = 2, kNotSpd = 3, kNonFinite = 4 };

// Packed-batch descriptor of one problem: shape and float offsets into each
// packed array kind (see SSPCG_ARRAY_* in sspcg.h).
struct ProbDesc {
  int32_t N, nx, nu, id;  // id: index of the problem in the caller's per-problem output arrays
  int64_t oA, oB, oq, orr, odiag, ooff, ovec;
};

// Problem set of a launch: either a device descriptor array (batched) or a
// single descriptor passed by value (single-problem calls; no device memory).
struct ProbSet {
  const ProbDesc *desc;  // device array of nprob descriptors, or nullptr
  ProbDesc single;       // used when desc == nullptr (problem 0)
  int32_t nprob;
  __device__ __forceinline__ ProbDesc get(int p) const { return desc ? desc[p] : single; }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2.  Error-free transformations after Knuth (TwoSum) and Dekker
// (Fast2Sum); the exact product uses one fused multiply-add.  About 48
// significant bits from FP32 units, which on this GPU run at 64x the FP64
// rate.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

// acc += a * b with the product formed exactly.
__device__ __forceinline__ df df_fma(df acc, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);
  df s = two_sum(acc.hi, p);
  float e = __fadd_rn(s.lo, __fadd_rn(acc.lo, pe));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_shfl_xor(df v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// Products of double-float values: the exact product of the high parts (one
// FMA gives its error) plus the cross terms; the lo * lo term is below the
// format's precision.
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// c + a * b for double-float a, b, c.
__device__ __forceinline__ df df_fma3(df a, df b, df c) {
  float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  df s = two_sum(c.hi, p);
  float e = __fadd_rn(s.lo, __fadd_rn(c.lo, pe));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// 1 / x: the FP32 reciprocal and one Newton step y + y (1 - x y) with the
// residual formed in double-float (about 46 bits).
__device__ __forceinline__ df df_rcp(df x) {
  const float y = __frcp_rn(x.hi);
  const df r = df_fma3(df_neg(x), df{y, 0.0f}, df{1.0f, 0.0f});  // 1 - x y
  return fast_two_sum(y, __fmul_rn(y, r.hi));
}

// sqrt(x), x > 0: the FP32 square root and one Newton step s + (x - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df x) {
  const float s = __fsqrt_rn(x.hi);
  const df r = df_fma3(df{-s, 0.0f}, df{s, 0.0f}, x);  // x - s^2
  return fast_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}

// Ceil-div helpers.
__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Find the problem owning global knot g: knot_start is an exclusive prefix
// of (N_i + 1) with nprob + 1 entries.
__device__ __forceinline__ int find_problem(const int64_t *knot_start, int nprob, int64_t g) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (knot_start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Host: set a kernel's largest dynamic shared memory once per device.  Bit d
// of ``done`` records device d; devices beyond 63 set it on every call.
template <typename Kern>
inline cudaError_t smem_attr_once(std::atomic<uint64_t> &done, Kern kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t{1} << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace sspcg
