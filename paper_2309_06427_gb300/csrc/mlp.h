// Host-side declarations of the warm-start network's kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sspcg {
namespace mlp {

// Feature row layout (columns of X): see the header comment of sspcg_mlp_* in sspcg.h.
constexpr int kIn = 1344, kHid = 256, kOut = 32;
constexpr int kPadX = 28, kPadU = 14;
constexpr int kOffA = 0, kOffB = 784, kOffQp = 1176, kOffRp = 1204, kOffQ = 1218, kOffG = 1246, kOffDj = 1274,
              kOffNx = 1302;
// Flat FP32 parameter layout: W1 [256][1344], b1, W2 [256][256], b2, W3 [32][256], b3.
constexpr int64_t kW1 = 0, kB1 = kW1 + (int64_t)kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + (int64_t)kHid * kHid,
                  kW3 = kB2 + kHid, kB3 = kW3 + (int64_t)kOut * kHid, kParams = kB3 + kOut;
// Weight-gradient products split their row contraction into at most kMaxSplits chunks of at least
// kRowsPerSplit rows, summed in a fixed order afterwards.
constexpr int kRowsPerSplit = 512;
constexpr int kMaxSplits = 64;

using bf16 = __nv_bfloat16;

// Knot rows [row0, row0 + nrows) of the batch (refs: (problem, block row) per knot).
struct RowSpan {
  ProbSet ps;
  const int2 *kref;
  int64_t row0, nrows;
};

struct QpData {
  const float *A, *B, *qd, *rd, *gamma, *PD;
};

// Gather table of the feature columns for every (nx <= 28, nu <= 14): kFeatTable int16 entries (host).
constexpr int64_t kFeatTable = (int64_t)kPadX * (kPadU + 1) * kIn;
void build_feature_table(int16_t *tab);
// Normalised bf16 feature rows of the span into X; tab: the gather table on the device.
cudaError_t launch_features(const RowSpan &rs, const QpData &q, const float *mu, const float *isd,
                            const int16_t *tab, bf16 *X, cudaStream_t st);
// Column sums of the raw features over the span: part [warps][2][kIn] (FP64); returns warps used.
cudaError_t launch_feature_stats(const RowSpan &rs, const QpData &q, double *part, int warps, cudaStream_t st);
cudaError_t launch_stats_finish(const double *part, int warps, int64_t rows, float *mu, float *isd,
                                cudaStream_t st);
int feature_stats_warps(int sms);

enum Epilogue : int { kEpiBiasRelu = 0, kEpiBiasF32 = 1, kEpiMask = 2 };
// C[M][N] = epilogue(A[M][K] B[N][K]^T) with bf16 operands and FP32 accumulation.
cudaError_t launch_gemm_nt(int epi, const bf16 *A, const bf16 *B, int64_t M, int N, int K, const float *bias,
                           const bf16 *mask, bf16 *Cb, float *Cf, cudaStream_t st);
// The same product on the 5th-generation tensor cores (tcgen05 + TMA): N in {256, 32}, K % 64 == 0,
// epilogues kEpiBiasRelu and kEpiBiasF32; *err is set to 1 when a bounded wait expires.
cudaError_t launch_gemm_nt_tc(int epi, const bf16 *A, const bf16 *B, int64_t M, int N, int K, const float *bias,
                              bf16 *Cb, float *Cf, int *err, cudaStream_t st);
// False when the driver's tensor-map encoder is unavailable.
bool tc_available();
// part[s][N1][N2] = sum over rows m of split s of G[m][n1] X[m][n2].
cudaError_t launch_gemm_tn(const bf16 *G, int N1, const bf16 *X, int N2, int64_t M, float *part, cudaStream_t st);
int64_t gemm_tn_splits(int64_t M);
// part[chunk][N] = column sums of Y[M][N] over the same row chunks as launch_gemm_tn.
cudaError_t launch_colsum(const bf16 *Y, int64_t M, int N, float *part, cudaStream_t st);
// out[i] = sum_s part[s][i], s in order.
cudaError_t launch_reduce_splits(const float *part, int64_t splits, int64_t n, float *out, cudaStream_t st);

// S^2-norm loss of problems [p0, p1) whose rows start at knot_start[p] - row0 in Y/U/dY.
struct LossArgs {
  ProbSet ps;
  int32_t p0, p1;
  const int64_t *knot_start;
  int64_t row0;
  const float *Y, *lamstar, *gamma, *D, *E;
  float *U;
  double *uu, *gg, *loss;
  bf16 *dY;
};
cudaError_t launch_loss(const LossArgs &a, cudaStream_t st);

// Adam on the flat parameters (update = false: only refresh the bf16 copies).
struct AdamArgs {
  float *w, *m, *v;
  const float *g;
  float lr, beta1, beta2, eps, bc1, bc2;
  int update;
  bf16 *W1b, *W2b, *W3b, *W2t, *W3t;
};
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st);

// lambda0 of rows [row0, row0 + nrows): lambda[ovec + k nx + i] = Y[r][i], i < nx.
cudaError_t launch_scatter_lambda(const RowSpan &rs, const float *Y, float *lambda, cudaStream_t st);

}  // namespace mlp
}  // namespace sspcg
