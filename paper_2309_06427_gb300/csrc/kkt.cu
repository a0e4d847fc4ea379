// The two outer steps of the Schur-complement method around the PCG solve
// (Eq. schur, Sec. II-A): the right-hand side gamma = c - C G^-1 g from the
// constraint values c and the cost gradient g = (q_0, r_0, ..., q_N), and
// the primal step delta z = G^-1 (g - C^T lambda*) = G^-1 (g + C^T mu) from
// the library's solution mu = -lambda*.  With the constraint rows -x_0 and
// A_k x_k + B_k u_k - x_{k+1} and G = blockdiag(diag qd_k, diag rd_k):
//   gamma_0     = c_0 + q_0 / qd_0
//   gamma_{k+1} = c_{k+1} - A_k (q_k / qd_k) - B_k (r_k / rd_k) + q_{k+1} / qd_{k+1}
//   dx_k = (q_k - mu_k + A_k^T mu_{k+1}) / qd_k   (no A term at k = N)
//   du_k = (r_k + B_k^T mu_{k+1}) / rd_k
// One warp per knot; lane i owns row i of the knot's block (nx, nu <= 28).
#include <algorithm>

#include "../../include/sspcg.h"
#include "common.cuh"
#include "host.h"

namespace sspcg {
namespace {

constexpr int kKktWarps = 8;

__global__ void __launch_bounds__(kKktWarps * 32)
    form_gamma_kernel(ProbSet ps, const int2 *refs, int64_t knots, const float *__restrict__ A,
                      const float *__restrict__ B, const float *__restrict__ qd, const float *__restrict__ rd,
                      const float *__restrict__ c, const float *__restrict__ q, const float *__restrict__ r,
                      float *__restrict__ gamma) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kKktWarps + (threadIdx.x >> 5);
  if (g >= knots) return;
  const int2 ref = refs ? refs[g] : make_int2(0, (int)g);
  const ProbDesc d = ps.get(ref.x);
  const int k = ref.y, m = d.nx, u = d.nu;
  // scaled gradient of knot k-1, one entry per lane (zero past the block)
  float sq = 0.f, sr = 0.f;
  if (k > 0) {
    if (lane < m) sq = q[d.ovec + (int64_t)(k - 1) * m + lane] / qd[d.oq + (int64_t)(k - 1) * m + lane];
    if (lane < u) sr = r[d.orr + (int64_t)(k - 1) * u + lane] / rd[d.orr + (int64_t)(k - 1) * u + lane];
  }
  float acc = 0.f;
  if (k > 0) {
    const float *Ar = A + d.oA + (int64_t)(k - 1) * m * m + (int64_t)(lane < m ? lane : 0) * m;
    for (int j = 0; j < m; ++j) {
      const float s = __shfl_sync(0xffffffffu, sq, j);
      if (lane < m) acc = fmaf(Ar[j], s, acc);
    }
    if (u > 0) {
      const float *Br = B + d.oB + (int64_t)(k - 1) * m * u + (int64_t)(lane < m ? lane : 0) * u;
      for (int j = 0; j < u; ++j) {
        const float s = __shfl_sync(0xffffffffu, sr, j);
        if (lane < m) acc = fmaf(Br[j], s, acc);
      }
    }
  }
  if (lane < m) {
    const int64_t e = d.ovec + (int64_t)k * m + lane;
    const float own = q[e] / qd[d.oq + (int64_t)k * m + lane];
    gamma[e] = k == 0 ? c[e] + own : c[e] - acc + own;
  }
}

__global__ void __launch_bounds__(kKktWarps * 32)
    recover_step_kernel(ProbSet ps, const int2 *refs, int64_t knots, const float *__restrict__ A,
                        const float *__restrict__ B, const float *__restrict__ qd, const float *__restrict__ rd,
                        const float *__restrict__ q, const float *__restrict__ r, const float *__restrict__ mu,
                        float *__restrict__ dx, float *__restrict__ du) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kKktWarps + (threadIdx.x >> 5);
  if (g >= knots) return;
  const int2 ref = refs ? refs[g] : make_int2(0, (int)g);
  const ProbDesc d = ps.get(ref.x);
  const int k = ref.y, m = d.nx, u = d.nu, N = d.N;
  // mu_{k+1}, one entry per lane
  const float mn = (k < N && lane < m) ? mu[d.ovec + (int64_t)(k + 1) * m + lane] : 0.f;
  float ax = 0.f, bu = 0.f;
  if (k < N) {
    const float *Ac = A + d.oA + (int64_t)k * m * m + (lane < m ? lane : 0);        // column lane of A_k
    const float *Bc = u > 0 ? B + d.oB + (int64_t)k * m * u + (lane < u ? lane : 0) : nullptr;  // of B_k
    for (int l = 0; l < m; ++l) {
      const float s = __shfl_sync(0xffffffffu, mn, l);
      if (lane < m) ax = fmaf(Ac[(int64_t)l * m], s, ax);
      if (lane < u) bu = fmaf(Bc[(int64_t)l * u], s, bu);
    }
  }
  if (lane < m) {
    const int64_t e = d.ovec + (int64_t)k * m + lane;
    dx[e] = (q[e] - mu[e] + ax) / qd[d.oq + (int64_t)k * m + lane];
  }
  if (k < N && lane < u) {
    const int64_t e = d.orr + (int64_t)k * u + lane;
    du[e] = (r[e] + bu) / rd[e];
  }
}

unsigned kkt_grid(int64_t knots) { return (unsigned)((knots + kKktWarps - 1) / kKktWarps); }

bool shape_ok(int N, int nx, int nu) {
  return N >= 0 && N <= SSPCG_MAX_N && nx >= 1 && nx <= SSPCG_MAX_NX && nu >= 0 && nu <= SSPCG_MAX_NX;
}

ProbDesc single(int N, int nx, int nu) {
  ProbDesc d{};
  d.N = N; d.nx = nx; d.nu = nu;
  return d;
}

}  // namespace
}  // namespace sspcg

using namespace sspcg;

#define KKT_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return sspcg::host::cuda_error(e_);  \
  } while (0)

extern "C" {

sspcg_status sspcg_form_gamma(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                              const float *rd, const float *c, const float *q, const float *r, float *gamma,
                              sspcg_stream stream) {
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!qd || !c || !q || !gamma || (N > 0 && (!A || (nu > 0 && (!B || !rd || !r))))) return SSPCG_ERR_INVALID_ARG;
  const int64_t knots = N + 1;
  form_gamma_kernel<<<kkt_grid(knots), kKktWarps * 32, 0, (cudaStream_t)stream>>>(
      ProbSet{nullptr, single(N, nx, nu), 1}, nullptr, knots, A, B, qd, rd, c, q, r, gamma);
  KKT_CUDA(cudaGetLastError());
  return SSPCG_OK;
}

sspcg_status sspcg_recover_step(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                                const float *rd, const float *q, const float *r, const float *mu, float *dx,
                                float *du, sspcg_stream stream) {
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!qd || !q || !mu || !dx || (N > 0 && (!A || (nu > 0 && (!B || !rd || !r || !du)))))
    return SSPCG_ERR_INVALID_ARG;
  const int64_t knots = N + 1;
  recover_step_kernel<<<kkt_grid(knots), kKktWarps * 32, 0, (cudaStream_t)stream>>>(
      ProbSet{nullptr, single(N, nx, nu), 1}, nullptr, knots, A, B, qd, rd, q, r, mu, dx, du);
  KKT_CUDA(cudaGetLastError());
  return SSPCG_OK;
}

sspcg_status sspcg_form_gamma_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                      const float *rd, const float *c, const float *q, const float *r, float *gamma,
                                      sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (v.nprob == 0) return SSPCG_OK;
  if (!qd || !c || !q || !gamma || (v.total_off > 0 && (!A || !B || !rd || !r))) return SSPCG_ERR_INVALID_ARG;
  form_gamma_kernel<<<kkt_grid(v.knots), kKktWarps * 32, 0, (cudaStream_t)stream>>>(v.ps, v.kref, v.knots, A, B, qd,
                                                                                   rd, c, q, r, gamma);
  KKT_CUDA(cudaGetLastError());
  return SSPCG_OK;
}

sspcg_status sspcg_recover_step_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                        const float *rd, const float *q, const float *r, const float *mu, float *dx,
                                        float *du, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (v.nprob == 0) return SSPCG_OK;
  if (!qd || !q || !mu || !dx || (v.total_off > 0 && (!A || !B || !rd || !r || !du))) return SSPCG_ERR_INVALID_ARG;
  recover_step_kernel<<<kkt_grid(v.knots), kKktWarps * 32, 0, (cudaStream_t)stream>>>(v.ps, v.kref, v.knots, A, B,
                                                                                     qd, rd, q, r, mu, dx, du);
  KKT_CUDA(cudaGetLastError());
  return SSPCG_OK;
}

}  // extern "C"
