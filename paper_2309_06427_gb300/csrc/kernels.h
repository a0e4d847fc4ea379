// Host-side declarations shared by the CUDA translation units of sspcg.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sspcg {

// Operator forms for S p.
enum OpForm : int { kOpBlock = 0, kOpQp = 1 };
// Precision of the dot-product reductions.
enum RedMode : int { kRedF32 = 0, kRedDf = 1, kRedF64 = 2 };

// Padded leading dimension of a matrix staged in shared memory: odd, so that
// 32 consecutive rows touch 32 distinct banks.
__host__ __device__ __forceinline__ int pad_ld(int x) { return x | 1; }

// Shared-memory carve-up of one PCG problem, in elements of the working
// precision; every region starts 16-byte aligned.  The first K block rows of
// the operator and preconditioner blocks are staged (K = N+1: fully
// resident; K = 0: everything read from L2/HBM each iteration).  The same
// function sizes launches on the host and carves on the device.
//
// Every vector has a zero segment before block row 0 and after block row N
// (the offsets below point at block row 0), so that a row's three block
// products read their neighbour segments without branches: the segment of
// the missing neighbour is zero.  A single-knot problem (N = 0) stages one
// zero off-diagonal slot, so that its clamped off-diagonal reads stay in
// bounds.
struct PcgLayout {
  int64_t p, r, w, x, e, u, s, v;   // vectors (e: the polynomial's residual; u, s: single-reduction CG)
  int64_t vu;                       // v_u block rows (QP form), after v_x
  int64_t iq, ir;                   // 1/q, 1/r (QP form)
  int64_t m0, m1, pd, pe;           // staged blocks
  int64_t total;
};

// Vectors are stored with a block-row stride of nx rounded up to 4 elements,
// so that every block row starts 16-byte aligned and a thread can load a
// whole block-row segment with 128-bit loads.
__host__ __device__ __forceinline__ int vec_stride(int x) { return (x + 3) & ~3; }

// Staged off-diagonal slots of a layout with K staged block rows: K (at most N), and one zero slot for N = 0.
__host__ __device__ __forceinline__ int64_t staged_off_slots(int K, int N) {
  const int64_t Ks = K < N ? K : N;
  return (N == 0 && K > 0) ? 1 : Ks;
}

__host__ __device__ inline PcgLayout pcg_layout(int op, int K, int N, int nx, int nu, int poly = 0, int cg = 0) {
  PcgLayout L{};
  const int64_t n = N + 1, NXP = vec_stride(nx), NUP = vec_stride(nu);
  const int64_t RVP = (n + 2) * NXP;  // a vector with its two zero segments
  const int64_t Ks = staged_off_slots(K, N);
  const int64_t ld = pad_ld(nx), ldb = pad_ld(nu > 0 ? nu : 1);
  int64_t o = 0;
  L.p = o + NXP; o += RVP;
  L.r = o + NXP; o += RVP;
  L.w = o + NXP; o += RVP;
  L.x = o + NXP; o += RVP;
  L.e = o + NXP;
  if (poly) o += RVP;
  L.u = o + NXP;
  if (cg) o += RVP;
  L.s = o + NXP;
  if (cg) o += RVP;
  L.v = o + NXP;  // the block form has no v (no region)
  L.vu = op == kOpQp ? L.v + (n + 1) * NXP + NUP : L.v;
  if (op == kOpQp) o += RVP + (int64_t)(N + 1) * NUP;   // v_x with its zero segments, then v_u after one
  L.iq = o;
  if (op == kOpQp) o += n * NXP;
  L.ir = o;
  if (op == kOpQp) o += (int64_t)N * NUP;
  if (op == kOpQp) {
    L.m0 = o; o += round_up(Ks * nx * ld, 4);    // A_k, row stride ld
    L.m1 = o; o += round_up(Ks * nx * ldb, 4);   // B_k, row stride ldb
  } else {
    L.m0 = o; o += round_up((int64_t)K * nx * ld, 4);  // D_k
    L.m1 = o; o += round_up(Ks * nx * ld, 4);          // E_k
  }
  L.pd = o; o += round_up((int64_t)K * nx * ld, 4);    // PD_k
  L.pe = o; o += round_up(Ks * nx * ld, 4);            // PE_k
  L.total = o;
  return L;
}

// Largest number of staged block rows whose layout fits in ``elems``; -1 when
// not even the vectors fit.
__host__ __device__ inline int pcg_max_resident(int op, int N, int nx, int nu, int64_t elems, int poly = 0,
                                                int cg = 0) {
  if (pcg_layout(op, N + 1, N, nx, nu, poly, cg).total <= elems) return N + 1;
  if (pcg_layout(op, 0, N, nx, nu, poly, cg).total > elems) return -1;
  int lo = 0, hi = N;  // invariant: layout(lo) fits, layout(hi + 1) does not
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (pcg_layout(op, mid, N, nx, nu, poly, cg).total <= elems) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Arguments of a PCG launch (by value).
struct PcgArgs {
  ProbSet ps;
  const int32_t *work;   // problem indices in processing order (device), or nullptr: identity
  int32_t nwork;
  int32_t *counter;      // work-queue counter (device, zeroed before launch), or nullptr: static
  const float *A, *B, *qd, *rd;  // QP operator data (packed, FP32)
  const float *D, *E;            // block operator data (packed, FP32)
  const void *PD, *PE;           // preconditioner blocks in the working precision
  const float *gamma;
  void *lambda;                  // solution: float when lambda_f32, else the working precision
  int32_t lambda_f32;
  int32_t *iters;
  double *relres;
  int32_t *status;       // in: nonzero skips the problem; out: solve code
  float tol2;            // tol^2
  int32_t max_iter;      // <= 0: 10 (N+1) nx
  int32_t warm;          // 0, 1, 2 (see sspcg_options)
  int32_t poly;          // degree d of the polynomial preconditioner sum_{j<=d} (I - Phi^-1 S)^j Phi^-1
  int32_t cg;            // 1: single-reduction (Chronopoulos-Gear) PCG (QP form, FP32, double-float sums)
  int64_t smem_elems;    // dynamic shared memory of the launch, in elements of the working precision
  int32_t max_resident;  // cap on staged block rows (a schedule override); large = no cap
  void *gscratch;        // vectors in global memory: CTA b uses gscratch + b * gstride elements
  int64_t gstride;       //   (nullptr: vectors in shared memory)
  int32_t warp;          // 1: one problem per warp (smem_elems per warp), QP form, textbook PCG
  const float *pad;      // padded copies of A, B, PE of the streamed problems (QP form, FP32), or nullptr
  const int64_t *pad_off;  // per problem id: offset of its copies in pad, or -1 (read the inputs)
};

// Floats of one padded region (rows of vec_stride(width) values), a multiple of 8 so that every region of a
// problem starts 32-byte aligned (the PCG reads padded rows of a multiple of 8 values with 256-bit loads).
__host__ __device__ __forceinline__ int64_t pad_region(int64_t rows, int width) {
  return round_up(rows * vec_stride(width), 8);
}

// Padded copies for the streamed block rows of the listed problems (desc indices): A_k and PE_k rows of
// vec_stride(nx) values, B_k rows of vec_stride(nu), zeros in the padding; problem p's copies start at
// pad_off[desc[p].id] (a multiple of 8 floats): A, then B at + pad_region(N nx, nx), then PE after B's
// pad_region(N nx, nu).  PE nullptr: no PE copy.
cudaError_t launch_pad_rows(const ProbDesc *desc, const int32_t *list, int32_t count, const float *A,
                            const float *B, const float *PE, const int64_t *pad_off, float *pad, int sms,
                            cudaStream_t st);

// PCG launch for one nx; dispatches to the instantiation for that nx.
// f64: the FP64 path (QP operator form only).  Each problem stages as many
// block rows as fit in ``smem`` bytes (at most a.max_resident).
cudaError_t launch_pcg(int nx, int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem,
                       cudaStream_t st);

int pcg_max_smem_bytes();
// CTAs of that PCG variant that fit on one SM at ``block`` threads and ``smem`` bytes of dynamic shared memory
// (registers, threads and shared memory; gv: vectors in a global workspace; cg: single-reduction PCG;
// warp: one problem per warp).
cudaError_t occupancy_pcg(int nx, int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem,
                          int *ctas);

// Schur build and preconditioner assembly; Real = float (FP32 blocks) or
// double (the FP64 path).  refs[i] = (problem, block row) of work item i
// (nullptr: one problem, item i is block row i, or i + 1 for off-diagonals).
// mx: the largest nx and nu of the launch (sizes the per-warp shared memory).
template <typename Real>
cudaError_t launch_schur_build(const ProbSet &ps, const int2 *refs, int64_t total_knots, const float *A,
                               const float *B, const float *qd, const float *rd, Real *D, Real *E,
                               cudaStream_t st, int sms, int mx);
// Schur blocks with full SPD cost blocks from their inverses: Qi laid out like
// D, R_{k-1}^-1 of problem p at roff[p] + (k-1) nu^2 (roff nullptr: offset 0).
cudaError_t launch_schur_full(const ProbSet &ps, const int2 *refs, int64_t total_knots, const int64_t *roff,
                              const float *A, const float *B, const float *Qi, const float *Ri, float *D, float *E,
                              cudaStream_t st, int mx);
// Diagonal blocks of Phi^-1 (FP64 inverses), one thread per knot: every
// knot of a launch must have the same nx.
template <typename Real>
cudaError_t launch_precond_inv(const ProbSet &ps, const int2 *refs, int64_t total_knots, int nx, int kind,
                               const Real *D, Real *PD, int32_t *status, cudaStream_t st);
// Off-diagonal blocks of Phi^-1 (any mix of nx).
template <typename Real>
cudaError_t launch_precond_off(const ProbSet &ps, const int2 *refs, int64_t total_off, int kind,
                               const Real *E, const Real *PD, Real *PE, cudaStream_t st, int sms, int64_t off_elems,
                               int mx);
cudaError_t launch_residual_qp(const ProbSet &ps, const float *A, const float *B, const float *qd, const float *rd,
                               const float *gamma, const float *lambda, double *relres_true, cudaStream_t st);

}  // namespace sspcg
