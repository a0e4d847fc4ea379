// Schur-block build (Sec. II-A) and preconditioner assembly (Eq. stair_inv,
// Sec. III, Sec. IV, Eq. jacobi).  One warp per knot; the batch is a flat
// list of knots, each warp finding its problem by binary search.
#include "common.cuh"
#include "kernels.h"

namespace sspcg {

constexpr int kBuildWarps = 4;  // warps per CTA of the build kernels

// ---------------------------------------------------------------------------
// K1: D_k, E_k from (A, B, diag Q, diag R).
//   D_0 = Q_0^-1
//   D_k = A_{k-1} Q_{k-1}^-1 A_{k-1}^T + B_{k-1} R_{k-1}^-1 B_{k-1}^T + Q_k^-1   (= -theta_{k-1})
//   E[k-1] = S(k, k-1) = -A_{k-1} Q_{k-1}^-1                                   (= -phi_{k-1})
// Real = float (FP32 arithmetic) or double (the FP64 path); only the upper
// triangle of D_k is summed and mirrored, so D_k is exactly symmetric.
// Shared memory per warp: AQ (nx*nx), A (nx*nx), BR (nx*nu), B (nx*nu), 1/q_k (nx).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kBuildWarps * 32) schur_build_kernel(ProbSet ps, const int64_t *knot_start,
                                                                      int64_t total_knots, const float *__restrict__ A,
                                                                      const float *__restrict__ B,
                                                                      const float *__restrict__ qd,
                                                                      const float *__restrict__ rd, Real *D, Real *E) {
  extern __shared__ float4 smem_raw[];
  Real *smem = reinterpret_cast<Real *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int per_warp = 2 * kMaxNx * kMaxNx + 2 * kMaxNx * kMaxNx + kMaxNx;
  Real *sAQ = smem + wid * per_warp;
  Real *sA = sAQ + kMaxNx * kMaxNx;
  Real *sBR = sA + kMaxNx * kMaxNx;
  Real *sB = sBR + kMaxNx * kMaxNx;
  Real *sIq = sB + kMaxNx * kMaxNx;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_knots; g += (int64_t)gridDim.x * kBuildWarps) {
    const int p = knot_start ? find_problem(knot_start, ps.nprob, g) : 0;
    const ProbDesc d = ps.get(p);
    const int k = (int)(g - (knot_start ? knot_start[p] : 0));
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
    for (int e = lane; e < nn; e += 32) {
      const int i = e / nx, j = e - i * nx;
      if (i > j) continue;
      Real s = Real(0);
      for (int l = 0; l < nx; ++l) s = fma(sAQ[i * nx + l], sA[j * nx + l], s);
      for (int m = 0; m < nu; ++m) s = fma(sBR[i * nu + m], sB[j * nu + m], s);
      if (i == j) s += sIq[i];
      Dk[i * nx + j] = s;
      Dk[j * nx + i] = s;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K2a: PD_k = D_k^-1.  FP64 LDL^T of the SPD block (no square roots), then
// D^-1 = L^-T diag(1/d) L^-1.  Lane i owns row i (nx <= 28 < 32).
// Reciprocals start from the FP32 reciprocal and take two Newton steps in
// FP64 (each doubles the correct bits: 2^-23 -> 2^-46 -> below 2^-53).
// Jacobi: PD_k = diag(1 / D_k(i,i)).
// Shared memory per warp: M (nx*nx doubles), W (nx*nx doubles), invd (nx doubles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_f64(double x) {
  double y = (double)(1.0f / (float)x);
  y = y * fma(-x, y, 2.0);
  y = y * fma(-x, y, 2.0);
  return y;
}

template <typename Real>
__global__ void __launch_bounds__(kBuildWarps * 32) precond_diag_kernel(ProbSet ps, const int64_t *knot_start,
                                                                       int64_t total_knots, int kind,
                                                                       const Real *__restrict__ D, Real *PD,
                                                                       int32_t *status) {
  extern __shared__ double dsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int per_warp = 2 * kMaxNx * kMaxNx + kMaxNx;
  double *M = dsm + wid * per_warp;
  double *W = M + kMaxNx * kMaxNx;
  double *invd = W + kMaxNx * kMaxNx;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_knots; g += (int64_t)gridDim.x * kBuildWarps) {
    const int p = knot_start ? find_problem(knot_start, ps.nprob, g) : 0;
    const ProbDesc d = ps.get(p);
    const int k = (int)(g - (knot_start ? knot_start[p] : 0));
    const int nx = d.nx, nn = nx * nx;
    const Real *Dk = D + d.odiag + (int64_t)k * nn;
    Real *PDk = PD + d.odiag + (int64_t)k * nn;
    if (kind == 3) {  // Jacobi
      bool bad = false;
      for (int e = lane; e < nn; e += 32) {
        const int i = e / nx, j = e - i * nx;
        Real v = Real(0);
        if (i == j) {
          const Real s = Dk[e];
          bad |= !(s > Real(0)) || !isfinite(s);
          v = Real(1) / s;
        }
        PDk[e] = v;
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) status[d.id] = kNotSpd;
      continue;
    }
    for (int e = lane; e < nn; e += 32) M[e] = (double)Dk[e];
    __syncwarp();
    // LDL^T, right-looking.  After step j: invd[j] = 1/d_j, M(i, j) = L(i, j) for i > j.
    bool ok = true;
    for (int j = 0; j < nx; ++j) {
      const double djj = M[j * nx + j];
      if (!(djj > 0.0) || !isfinite(djj)) { ok = false; break; }
      const double inv = rcp_f64(djj);
      double uij = 0.0;  // unscaled column value M(i, j) of this lane's row
      if (lane > j && lane < nx) uij = M[lane * nx + j];
      __syncwarp();
      if (lane > j && lane < nx) {
        const double lij = uij * inv;
        // trailing update of row `lane`, columns j+1..lane: M(i,c) -= L(i,j) * u(c,j)
        for (int c = j + 1; c <= lane; ++c) M[lane * nx + c] -= lij * M[c * nx + j];
      }
      __syncwarp();
      if (lane > j && lane < nx) M[lane * nx + j] = uij * inv;
      if (lane == 0) invd[j] = inv;
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) status[d.id] = kNotSpd;
      for (int e = lane; e < nn; e += 32) PDk[e] = Real(0);
      __syncwarp();
      continue;
    }
    // W = L^-1 (unit lower): lane c computes column c by forward substitution.
    if (lane < nx) {
      const int c = lane;
      for (int i = 0; i < nx; ++i) {
        double v = 0.0;
        if (i == c) v = 1.0;
        else if (i > c) {
          for (int t = c; t < i; ++t) v -= M[i * nx + t] * W[t * nx + c];
        }
        W[i * nx + c] = v;
      }
    }
    __syncwarp();
    // D^-1(i, j) = sum_{t >= max(i,j)} W(t, i) W(t, j) / d_t; lane i computes j >= i and mirrors.
    if (lane < nx) {
      const int i = lane;
      for (int j = i; j < nx; ++j) {
        double s = 0.0;
        for (int t = j; t < nx; ++t) s += W[t * nx + i] * W[t * nx + j] * invd[t];
        const Real f = (Real)s;
        PDk[i * nx + j] = f;
        PDk[j * nx + i] = f;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// K2b: PE[k-1] = -c * PD_k E[k-1] PD_{k-1}, c = 1 (symmetric stair) or 1/2
// (additive stair), in Real.  One warp per off-diagonal block.
// Shared memory per warp: PD_k, E, PD_{k-1}, T = PD_k E (4 * nx * nx floats).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kBuildWarps * 32) precond_off_kernel(ProbSet ps, const int64_t *off_start,
                                                                      int64_t total_off, Real c,
                                                                      const Real *__restrict__ E,
                                                                      const Real *__restrict__ PD, Real *PE) {
  extern __shared__ float4 smem_raw[];
  Real *smem = reinterpret_cast<Real *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int per_warp = 4 * kMaxNx * kMaxNx;
  Real *sP1 = smem + wid * per_warp;
  Real *sE = sP1 + kMaxNx * kMaxNx;
  Real *sP0 = sE + kMaxNx * kMaxNx;
  Real *sT = sP0 + kMaxNx * kMaxNx;
  for (int64_t g = (int64_t)blockIdx.x * kBuildWarps + wid; g < total_off; g += (int64_t)gridDim.x * kBuildWarps) {
    const int p = off_start ? find_problem(off_start, ps.nprob, g) : 0;
    const ProbDesc d = ps.get(p);
    const int k = 1 + (int)(g - (off_start ? off_start[p] : 0));  // block row k >= 1
    const int nx = d.nx, nn = nx * nx;
    const Real *P1 = PD + d.odiag + (int64_t)k * nn;
    const Real *P0 = PD + d.odiag + (int64_t)(k - 1) * nn;
    const Real *Ek = E + d.ooff + (int64_t)(k - 1) * nn;
    Real *PEk = PE + d.ooff + (int64_t)(k - 1) * nn;
    for (int e = lane; e < nn; e += 32) {
      sP1[e] = P1[e];
      sE[e] = Ek[e];
      sP0[e] = P0[e];
    }
    __syncwarp();
    for (int e = lane; e < nn; e += 32) {
      const int i = e / nx, j = e - i * nx;
      Real s = Real(0);
      for (int t = 0; t < nx; ++t) s = fma(sP1[i * nx + t], sE[t * nx + j], s);
      sT[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < nn; e += 32) {
      const int i = e / nx, j = e - i * nx;
      Real s = Real(0);
      for (int t = 0; t < nx; ++t) s = fma(sT[i * nx + t], sP0[t * nx + j], s);
      PEk[e] = -c * s;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
static int build_grid(int64_t items, int sms) {
  const int64_t need = cdiv(items, kBuildWarps);
  const int64_t cap = (int64_t)sms * 8;
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

template <typename Real>
cudaError_t launch_schur_build(const ProbSet &ps, const int64_t *knot_start, int64_t total_knots, const float *A,
                               const float *B, const float *qd, const float *rd, Real *D, Real *E,
                               cudaStream_t st, int sms) {
  if (total_knots == 0) return cudaSuccess;
  const size_t smem = sizeof(Real) * kBuildWarps * (4 * kMaxNx * kMaxNx + kMaxNx);
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(schur_build_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  schur_build_kernel<Real><<<build_grid(total_knots, sms), kBuildWarps * 32, smem, st>>>(ps, knot_start, total_knots,
                                                                                          A, B, qd, rd, D, E);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_precond_build(const ProbSet &ps, const int64_t *knot_start, int64_t total_knots,
                                 const int64_t *off_start, int64_t total_off, int kind, const Real *D,
                                 const Real *E, Real *PD, Real *PE, int32_t *status, cudaStream_t st, int sms,
                                 int64_t off_elems) {
  if (total_knots == 0) return cudaSuccess;
  const size_t smem_d = sizeof(double) * kBuildWarps * (2 * kMaxNx * kMaxNx + kMaxNx);
  const size_t smem_o = sizeof(Real) * kBuildWarps * (4 * kMaxNx * kMaxNx);
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(precond_diag_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(precond_off_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_o);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  precond_diag_kernel<Real><<<build_grid(total_knots, sms), kBuildWarps * 32, smem_d, st>>>(ps, knot_start,
                                                                                             total_knots, kind, D, PD,
                                                                                             status);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (total_off == 0) return cudaSuccess;
  if (kind == 2 || kind == 3) {  // block-Jacobi, Jacobi: no off-diagonal blocks
    return cudaMemsetAsync(PE, 0, sizeof(Real) * off_elems, st);
  }
  const Real c = (kind == 0) ? Real(1) : Real(0.5);
  precond_off_kernel<Real><<<build_grid(total_off, sms), kBuildWarps * 32, smem_o, st>>>(ps, off_start, total_off, c,
                                                                                          E, PD, PE);
  return cudaGetLastError();
}

template cudaError_t launch_schur_build<float>(const ProbSet &, const int64_t *, int64_t, const float *, const float *,
                                               const float *, const float *, float *, float *, cudaStream_t, int);
template cudaError_t launch_schur_build<double>(const ProbSet &, const int64_t *, int64_t, const float *,
                                                const float *, const float *, const float *, double *, double *,
                                                cudaStream_t, int);
template cudaError_t launch_precond_build<float>(const ProbSet &, const int64_t *, int64_t, const int64_t *, int64_t,
                                                 int, const float *, const float *, float *, float *, int32_t *,
                                                 cudaStream_t, int, int64_t);
template cudaError_t launch_precond_build<double>(const ProbSet &, const int64_t *, int64_t, const int64_t *,
                                                  int64_t, int, const double *, const double *, double *, double *,
                                                  int32_t *, cudaStream_t, int, int64_t);

}  // namespace sspcg
