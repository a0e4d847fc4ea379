// True residual ||gamma - S lambda||_2 / ||gamma||_2 in FP64 with S applied in
// the factored form of Eq. (schur), S = C G^-1 C^T, from the QP data.
// Diagnostic: one CTA per problem, block rows processed in chunks whose
// v = G^-1 C^T lambda values live in shared memory.
#include "common.cuh"
#include "kernels.h"

namespace sspcg {

constexpr int kResThreads = 256;
constexpr int kResChunk = 32;  // block rows per chunk

__global__ void __launch_bounds__(kResThreads) residual_qp_kernel(ProbSet ps, const float *__restrict__ A,
                                                                  const float *__restrict__ B,
                                                                  const float *__restrict__ qd,
                                                                  const float *__restrict__ rd,
                                                                  const float *__restrict__ gamma,
                                                                  const float *__restrict__ lambda, double *out) {
  __shared__ double vx[(kResChunk + 1) * kMaxNx];
  __shared__ double vu[(kResChunk + 1) * kMaxNx];
  __shared__ double red[2][kResThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int p = blockIdx.x; p < ps.nprob; p += gridDim.x) {
    const ProbDesc d = ps.get(p);
    const int N = d.N, nx = d.nx, nu = d.nu;
    const float *Ap = A + d.oA, *Bp = B + d.oB, *q = qd + d.oq, *r = rd + d.orr;
    const float *g = gamma + d.ovec, *x = lambda + d.ovec;
    double res2 = 0.0, g2 = 0.0;
    for (int k0 = 0; k0 <= N; k0 += kResChunk) {
      const int k1 = min(N + 1, k0 + kResChunk);
      const int kb = k0 > 0 ? k0 - 1 : 0;  // first knot whose v is needed
      // v_x(k)[j] = (-x_k[j] + sum_l A_k[l][j] x_{k+1}[l]) / q_k[j];  v_u(k)[j] = sum_l B_k[l][j] x_{k+1}[l] / r_k[j]
      for (int e = tid; e < (k1 - kb) * (nx + nu); e += kResThreads) {
        const int kk = e / (nx + nu), c = e - kk * (nx + nu), k = kb + kk;
        if (c < nx) {
          double s = -(double)x[k * nx + c];
          if (k < N)
            for (int l = 0; l < nx; ++l)
              s += (double)Ap[((int64_t)k * nx + l) * nx + c] * (double)x[(k + 1) * nx + l];
          vx[kk * kMaxNx + c] = s / (double)q[k * nx + c];
        } else if (k < N) {
          const int j = c - nx;
          double s = 0.0;
          for (int l = 0; l < nx; ++l) s += (double)Bp[((int64_t)k * nx + l) * nu + j] * (double)x[(k + 1) * nx + l];
          vu[kk * kMaxNx + j] = s / (double)r[k * nu + j];
        }
      }
      __syncthreads();
      // (S x)_k[i] = -v_x(k)[i] + A_{k-1}[i,:] v_x(k-1) + B_{k-1}[i,:] v_u(k-1)
      for (int e = tid; e < (k1 - k0) * nx; e += kResThreads) {
        const int k = k0 + e / nx, i = e % nx, kk = k - kb;
        double s = -vx[kk * kMaxNx + i];
        if (k > 0) {
          for (int j = 0; j < nx; ++j) s += (double)Ap[((int64_t)(k - 1) * nx + i) * nx + j] * vx[(kk - 1) * kMaxNx + j];
          for (int j = 0; j < nu; ++j) s += (double)Bp[((int64_t)(k - 1) * nx + i) * nu + j] * vu[(kk - 1) * kMaxNx + j];
        }
        const double gi = (double)g[k * nx + i];
        const double ri = gi - s;
        res2 += ri * ri;
        g2 += gi * gi;
      }
      __syncthreads();
    }
    res2 = warp_sum(res2);
    g2 = warp_sum(g2);
    if (lane == 0) { red[0][wid] = res2; red[1][wid] = g2; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kResThreads / 32; ++w) { a += red[0][w]; b += red[1][w]; }
      out[d.id] = b > 0.0 ? sqrt(a / b) : 0.0;
    }
    __syncthreads();
  }
}

cudaError_t launch_residual_qp(const ProbSet &ps, const float *A, const float *B, const float *qd, const float *rd,
                               const float *gamma, const float *lambda, double *relres_true, cudaStream_t st) {
  if (ps.nprob == 0) return cudaSuccess;
  const int grid = ps.nprob < 4096 ? ps.nprob : 4096;
  residual_qp_kernel<<<grid, kResThreads, 0, st>>>(ps, A, B, qd, rd, gamma, lambda, relres_true);
  return cudaGetLastError();
}

}  // namespace sspcg
