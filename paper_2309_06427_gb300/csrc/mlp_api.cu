// C ABI of the learned warm start: the network object, feature
// normalisation, inference, one training step, and the warm-started pipeline.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sspcg.h"
#include "host.h"
#include "mlp.h"

using namespace sspcg;
using namespace sspcg::mlp;

static_assert(kParams == SSPCG_MLP_PARAMS, "parameter count");
static_assert(kIn == SSPCG_MLP_IN && kHid == SSPCG_MLP_HIDDEN && kOut == SSPCG_MLP_OUT, "layer sizes");

struct sspcg_mlp {
  int32_t max_rows = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 [kParams]
  bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2t = nullptr, *W3t = nullptr;
  float *mu = nullptr, *isd = nullptr;  // [kIn]
  int16_t *ftab = nullptr;              // feature gather table [kFeatTable]
  int64_t t = 0;                        // Adam steps taken
  // workspace for max_rows rows
  bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dH2 = nullptr, *dH1 = nullptr;
  float *Y = nullptr, *U = nullptr;
  double *uu = nullptr, *gg = nullptr;
  float *part = nullptr;  // split partial sums of the gradient products
  double *stat_part = nullptr;
  int stat_warps = 0;
  int engine = SSPCG_MLP_ENGINE_TCGEN05;
  int *err = nullptr;  // device: set by a tensor-core product whose bounded wait expired
};

namespace {

#define MLP_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return sspcg::host::cuda_error(e_);  \
  } while (0)

void mlp_free(sspcg_mlp *n) {
  if (!n) return;
  for (void *p : {(void *)n->w, (void *)n->g, (void *)n->m, (void *)n->v, (void *)n->W1b, (void *)n->W2b,
                  (void *)n->W3b, (void *)n->W2t, (void *)n->W3t, (void *)n->mu, (void *)n->isd, (void *)n->X,
                  (void *)n->H1, (void *)n->H2, (void *)n->dY, (void *)n->dH2, (void *)n->dH1, (void *)n->Y,
                  (void *)n->U, (void *)n->uu, (void *)n->gg, (void *)n->part, (void *)n->stat_part, (void *)n->err,
                  (void *)n->ftab})
    cudaFree(p);
  delete n;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

QpData qp(const float *A, const float *B, const float *qd, const float *rd, const float *gamma, const float *PD) {
  return QpData{A, B, qd, rd, gamma, PD};
}

// The feature layout pads A_k to 28 x 28 and B_k to 28 x 14: batches with nu > 14 are not supported.
bool layout_fits(const host::PlanView &v) { return v.max_nu <= kPadU; }

bool qp_ok(const host::PlanView &v, const float *A, const float *B, const float *qd, const float *rd,
           const float *gamma, const float *PD) {
  if (!qd || !gamma || !PD) return false;
  if (v.total_off > 0 && (!A || !rd || !B)) return false;
  return true;
}

// Largest weight-gradient partial buffer: splits x max(W1 size, bias sizes).
int64_t part_floats(int64_t rows) { return gemm_tn_splits(rows) * (int64_t)kHid * kIn; }

sspcg_status refresh_copies(sspcg_mlp *n, cudaStream_t st) {
  AdamArgs a{};
  a.w = n->w; a.m = n->m; a.v = n->v; a.g = n->g;
  a.update = 0;
  a.W1b = n->W1b; a.W2b = n->W2b; a.W3b = n->W3b; a.W2t = n->W2t; a.W3t = n->W3t;
  MLP_CUDA(launch_adam(a, st));
  return SSPCG_OK;
}

// Forward over rows [row0, row0 + rows) of the plan: X, H1, H2, Y in the workspace.
sspcg_status forward(sspcg_mlp *n, const host::PlanView &v, int64_t row0, int64_t rows, const QpData &q,
                     cudaStream_t st) {
  RowSpan rs{v.ps, v.kref, row0, rows};
  MLP_CUDA(launch_features(rs, q, n->mu, n->isd, n->ftab, n->X, st));
  if (n->engine == SSPCG_MLP_ENGINE_TCGEN05) {
    MLP_CUDA(launch_gemm_nt_tc(kEpiBiasRelu, n->X, n->W1b, rows, kHid, kIn, n->w + kB1, n->H1, nullptr, n->err, st));
    MLP_CUDA(launch_gemm_nt_tc(kEpiBiasRelu, n->H1, n->W2b, rows, kHid, kHid, n->w + kB2, n->H2, nullptr, n->err, st));
    MLP_CUDA(launch_gemm_nt_tc(kEpiBiasF32, n->H2, n->W3b, rows, kOut, kHid, n->w + kB3, nullptr, n->Y, n->err, st));
    return SSPCG_OK;
  }
  MLP_CUDA(launch_gemm_nt(kEpiBiasRelu, n->X, n->W1b, rows, kHid, kIn, n->w + kB1, nullptr, n->H1, nullptr, st));
  MLP_CUDA(launch_gemm_nt(kEpiBiasRelu, n->H1, n->W2b, rows, kHid, kHid, n->w + kB2, nullptr, n->H2, nullptr, st));
  MLP_CUDA(launch_gemm_nt(kEpiBiasF32, n->H2, n->W3b, rows, kOut, kHid, n->w + kB3, nullptr, nullptr, n->Y, st));
  return SSPCG_OK;
}

// Weight and bias gradients of one layer: dW[N1][N2] = G^T X, db = column sums of G.
sspcg_status layer_grads(sspcg_mlp *n, const bf16 *G, int N1, const bf16 *Xin, int N2, int64_t rows, float *dW,
                         float *db, cudaStream_t st) {
  const int64_t splits = gemm_tn_splits(rows);
  MLP_CUDA(launch_gemm_tn(G, N1, Xin, N2, rows, n->part, st));
  MLP_CUDA(launch_reduce_splits(n->part, splits, (int64_t)N1 * N2, dW, st));
  MLP_CUDA(launch_colsum(G, rows, N1, n->part, st));
  MLP_CUDA(launch_reduce_splits(n->part, splits, N1, db, st));
  return SSPCG_OK;
}

}  // namespace

extern "C" {

sspcg_status sspcg_mlp_create(sspcg_mlp **out, int32_t max_rows) {
  if (!out || max_rows < 1) return SSPCG_ERR_INVALID_ARG;
  *out = nullptr;
  sspcg_mlp *n = new sspcg_mlp();
  n->max_rows = max_rows;
  const int64_t R = max_rows;
  auto fail = [&](cudaError_t e) { mlp_free(n); return sspcg::host::cuda_error(e); };
  cudaError_t e = cudaSuccess;
  auto alloc = [&](auto **p, int64_t count) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(**p) * std::max<int64_t>(count, 1));
  };
  alloc(&n->w, kParams); alloc(&n->g, kParams); alloc(&n->m, kParams); alloc(&n->v, kParams);
  alloc(&n->W1b, (int64_t)kHid * kIn); alloc(&n->W2b, (int64_t)kHid * kHid); alloc(&n->W3b, (int64_t)kOut * kHid);
  alloc(&n->W2t, (int64_t)kHid * kHid); alloc(&n->W3t, (int64_t)kHid * kOut);
  alloc(&n->mu, kIn); alloc(&n->isd, kIn);
  alloc(&n->X, R * kIn); alloc(&n->H1, R * kHid); alloc(&n->H2, R * kHid);
  alloc(&n->dY, R * kOut); alloc(&n->dH2, R * kHid); alloc(&n->dH1, R * kHid);
  alloc(&n->Y, R * kOut); alloc(&n->U, R * kOut);
  alloc(&n->uu, R); alloc(&n->gg, R);
  alloc(&n->part, part_floats(R));
  alloc(&n->err, 1);
  alloc(&n->ftab, kFeatTable);
  if (e != cudaSuccess) return fail(e);
  {
    std::vector<int16_t> tab(kFeatTable);
    build_feature_table(tab.data());
    if ((e = cudaMemcpy(n->ftab, tab.data(), sizeof(int16_t) * kFeatTable, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e);
  }
  if ((e = cudaMemset(n->err, 0, sizeof(int))) != cudaSuccess) return fail(e);
  if (!tc_available()) n->engine = SSPCG_MLP_ENGINE_MMA_SYNC;
  for (float *p : {n->w, n->g, n->m, n->v})
    if ((e = cudaMemset(p, 0, sizeof(float) * kParams)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(n->mu, 0, sizeof(float) * kIn)) != cudaSuccess) return fail(e);
  std::vector<float> ones(kIn, 1.0f);
  if ((e = cudaMemcpy(n->isd, ones.data(), sizeof(float) * kIn, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e);
  if (refresh_copies(n, nullptr) != SSPCG_OK) { mlp_free(n); return SSPCG_ERR_CUDA; }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  *out = n;
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_destroy(sspcg_mlp *mlp) {
  mlp_free(mlp);
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_set_engine(sspcg_mlp *n, int32_t engine) {
  if (!n || (engine != SSPCG_MLP_ENGINE_TCGEN05 && engine != SSPCG_MLP_ENGINE_MMA_SYNC)) return SSPCG_ERR_INVALID_ARG;
  if (engine == SSPCG_MLP_ENGINE_TCGEN05 && !tc_available()) return SSPCG_ERR_UNSUPPORTED;
  n->engine = engine;
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_status(const sspcg_mlp *n, int32_t *flag) {
  if (!n || !flag) return SSPCG_ERR_INVALID_ARG;
  int v = 0;
  MLP_CUDA(cudaMemcpy(&v, n->err, sizeof(int), cudaMemcpyDeviceToHost));
  *flag = v;
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_set_params(sspcg_mlp *n, const float *params, sspcg_stream stream) {
  if (!n || !params) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_CUDA(cudaMemcpyAsync(n->w, params, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, st));
  MLP_CUDA(cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, st));
  MLP_CUDA(cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, st));
  MLP_CUDA(cudaMemsetAsync(n->g, 0, sizeof(float) * kParams, st));
  n->t = 0;
  return refresh_copies(n, st);
}

sspcg_status sspcg_mlp_get_params(const sspcg_mlp *n, float *params, sspcg_stream stream) {
  if (!n || !params) return SSPCG_ERR_INVALID_ARG;
  MLP_CUDA(cudaMemcpyAsync(params, n->w, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_get_grads(const sspcg_mlp *n, float *grads, sspcg_stream stream) {
  if (!n || !grads) return SSPCG_ERR_INVALID_ARG;
  MLP_CUDA(cudaMemcpyAsync(grads, n->g, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_set_normalisation(sspcg_mlp *n, const float *mu, const float *inv_sigma,
                                         sspcg_stream stream) {
  if (!n || !mu || !inv_sigma) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_CUDA(cudaMemcpyAsync(n->mu, mu, sizeof(float) * kIn, cudaMemcpyDeviceToDevice, st));
  MLP_CUDA(cudaMemcpyAsync(n->isd, inv_sigma, sizeof(float) * kIn, cudaMemcpyDeviceToDevice, st));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_get_normalisation(const sspcg_mlp *n, float *mu, float *inv_sigma, sspcg_stream stream) {
  if (!n || !mu || !inv_sigma) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_CUDA(cudaMemcpyAsync(mu, n->mu, sizeof(float) * kIn, cudaMemcpyDeviceToDevice, st));
  MLP_CUDA(cudaMemcpyAsync(inv_sigma, n->isd, sizeof(float) * kIn, cudaMemcpyDeviceToDevice, st));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_fit_normalisation(sspcg_mlp *n, const sspcg_plan *plan, const float *A, const float *B,
                                         const float *qd, const float *rd, const float *gamma, const float *PD,
                                         sspcg_stream stream) {
  if (!n || !plan) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (v.nprob == 0) return SSPCG_OK;
  if (!qp_ok(v, A, B, qd, rd, gamma, PD)) return SSPCG_ERR_INVALID_ARG;
  if (!layout_fits(v)) return SSPCG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const int warps = feature_stats_warps(host::sms());
  if (n->stat_warps < warps) {
    cudaFree(n->stat_part);
    n->stat_part = nullptr;
    n->stat_warps = 0;
    MLP_CUDA(cudaMalloc(&n->stat_part, sizeof(double) * 2 * kIn * warps));
    n->stat_warps = warps;
  }
  RowSpan rs{v.ps, v.kref, 0, v.knots};
  MLP_CUDA(launch_feature_stats(rs, qp(A, B, qd, rd, gamma, PD), n->stat_part, warps, st));
  MLP_CUDA(launch_stats_finish(n->stat_part, warps, v.knots, n->mu, n->isd, st));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_features(const sspcg_mlp *n, const sspcg_plan *plan, int32_t p_begin, int32_t p_end,
                                const float *A, const float *B, const float *qd, const float *rd,
                                const float *gamma, const float *PD, uint16_t *X, sspcg_stream stream) {
  if (!n || !plan || !X) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (p_begin < 0 || p_end > v.nprob || p_begin > p_end) return SSPCG_ERR_INVALID_ARG;
  if (p_begin == p_end) return SSPCG_OK;
  if (!qp_ok(v, A, B, qd, rd, gamma, PD)) return SSPCG_ERR_INVALID_ARG;
  if (!layout_fits(v)) return SSPCG_ERR_UNSUPPORTED;
  const int64_t row0 = v.knot_start[p_begin], rows = v.knot_start[p_end] - row0;
  if (rows > n->max_rows) return SSPCG_ERR_INVALID_ARG;
  RowSpan rs{v.ps, v.kref, row0, rows};
  MLP_CUDA(launch_features(rs, qp(A, B, qd, rd, gamma, PD), n->mu, n->isd, n->ftab, reinterpret_cast<bf16 *>(X),
                           (cudaStream_t)stream));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_infer(sspcg_mlp *n, const sspcg_plan *plan, const float *A, const float *B,
                             const float *qd, const float *rd, const float *gamma, const float *PD, float *lambda0,
                             sspcg_stream stream) {
  if (!n || !plan || !lambda0) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (v.nprob == 0) return SSPCG_OK;
  if (!qp_ok(v, A, B, qd, rd, gamma, PD)) return SSPCG_ERR_INVALID_ARG;
  if (!layout_fits(v)) return SSPCG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const QpData q = qp(A, B, qd, rd, gamma, PD);
  for (int64_t r0 = 0; r0 < v.knots; r0 += n->max_rows) {
    const int64_t rows = std::min<int64_t>(n->max_rows, v.knots - r0);
    sspcg_status s = forward(n, v, r0, rows, q, st);
    if (s != SSPCG_OK) return s;
    MLP_CUDA(launch_scatter_lambda(RowSpan{v.ps, v.kref, r0, rows}, n->Y, lambda0, st));
  }
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_train_step(sspcg_mlp *n, const sspcg_plan *plan, int32_t p_begin, int32_t p_end,
                                  const float *A, const float *B, const float *qd, const float *rd,
                                  const float *gamma, const float *D, const float *E, const float *PD,
                                  const float *lambda_star, const sspcg_adam *hyper, double *loss,
                                  sspcg_stream stream) {
  if (!n || !plan || !hyper || !loss || !D || !lambda_star) return SSPCG_ERR_INVALID_ARG;
  const host::PlanView v = host::plan_view(plan);
  if (p_begin < 0 || p_end > v.nprob || p_begin >= p_end) return SSPCG_ERR_INVALID_ARG;
  if (!qp_ok(v, A, B, qd, rd, gamma, PD) || (v.total_off > 0 && !E)) return SSPCG_ERR_INVALID_ARG;
  if (!layout_fits(v)) return SSPCG_ERR_UNSUPPORTED;
  if (!(hyper->lr >= 0.f) || !(hyper->beta1 >= 0.f && hyper->beta1 < 1.f) ||
      !(hyper->beta2 >= 0.f && hyper->beta2 < 1.f) || !(hyper->eps > 0.f))
    return SSPCG_ERR_INVALID_ARG;
  const int64_t row0 = v.knot_start[p_begin], rows = v.knot_start[p_end] - row0;
  if (rows > n->max_rows) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  sspcg_status s = forward(n, v, row0, rows, qp(A, B, qd, rd, gamma, PD), st);
  if (s != SSPCG_OK) return s;
  LossArgs la{};
  la.ps = v.ps;
  la.p0 = p_begin;
  la.p1 = p_end;
  la.knot_start = v.d_knot_start;
  la.row0 = row0;
  la.Y = n->Y; la.lamstar = lambda_star; la.gamma = gamma; la.D = D; la.E = E;
  la.U = n->U; la.uu = n->uu; la.gg = n->gg; la.loss = loss; la.dY = n->dY;
  MLP_CUDA(launch_loss(la, st));
  // backward: output layer, then the two hidden layers (ReLU masks from the stored activations)
  if ((s = layer_grads(n, n->dY, kOut, n->H2, kHid, rows, n->g + kW3, n->g + kB3, st)) != SSPCG_OK) return s;
  MLP_CUDA(launch_gemm_nt(kEpiMask, n->dY, n->W3t, rows, kHid, kOut, nullptr, n->H2, n->dH2, nullptr, st));
  if ((s = layer_grads(n, n->dH2, kHid, n->H1, kHid, rows, n->g + kW2, n->g + kB2, st)) != SSPCG_OK) return s;
  MLP_CUDA(launch_gemm_nt(kEpiMask, n->dH2, n->W2t, rows, kHid, kHid, nullptr, n->H1, n->dH1, nullptr, st));
  if ((s = layer_grads(n, n->dH1, kHid, n->X, kIn, rows, n->g + kW1, n->g + kB1, st)) != SSPCG_OK) return s;
  // Adam
  n->t += 1;
  AdamArgs a{};
  a.w = n->w; a.m = n->m; a.v = n->v; a.g = n->g;
  a.lr = hyper->lr; a.beta1 = hyper->beta1; a.beta2 = hyper->beta2; a.eps = hyper->eps;
  a.bc1 = (float)(1.0 - std::pow((double)hyper->beta1, (double)n->t));
  a.bc2 = (float)(1.0 - std::pow((double)hyper->beta2, (double)n->t));
  a.update = 1;
  a.W1b = n->W1b; a.W2b = n->W2b; a.W3b = n->W3b; a.W2t = n->W2t; a.W3t = n->W3t;
  MLP_CUDA(launch_adam(a, st));
  return SSPCG_OK;
}

// Checkpoint blob: a header, then the FP32 parameters (the masters), Adam's first and second moments, and
// the feature normalisation (mu, 1/sigma).  The bf16 weight copies are derived from the masters.
namespace {
struct CkptHeader {
  char magic[8];  // "SSPCGMLP"
  int32_t version, in, hidden, out;
  int64_t params, steps;
};
constexpr int32_t kCkptVersion = 1;
constexpr int64_t kCkptBytes = (int64_t)sizeof(CkptHeader) + 3 * kParams * (int64_t)sizeof(float) +
                               2 * (int64_t)kIn * (int64_t)sizeof(float);
}  // namespace

sspcg_status sspcg_mlp_checkpoint_bytes(int64_t *bytes) {
  if (!bytes) return SSPCG_ERR_INVALID_ARG;
  *bytes = kCkptBytes;
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_save(const sspcg_mlp *n, void *host_buf, int64_t bytes, sspcg_stream stream) {
  if (!n || !host_buf || bytes < kCkptBytes) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CkptHeader h{};
  std::memcpy(h.magic, "SSPCGMLP", 8);
  h.version = kCkptVersion; h.in = kIn; h.hidden = kHid; h.out = kOut; h.params = kParams; h.steps = n->t;
  char *b = static_cast<char *>(host_buf);
  std::memcpy(b, &h, sizeof(h));
  char *cur = b + sizeof(h);
  for (const float *src : {(const float *)n->w, (const float *)n->m, (const float *)n->v}) {
    MLP_CUDA(cudaMemcpyAsync(cur, src, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
    cur += sizeof(float) * kParams;
  }
  for (const float *src : {(const float *)n->mu, (const float *)n->isd}) {
    MLP_CUDA(cudaMemcpyAsync(cur, src, sizeof(float) * kIn, cudaMemcpyDeviceToHost, st));
    cur += sizeof(float) * kIn;
  }
  MLP_CUDA(cudaStreamSynchronize(st));
  return SSPCG_OK;
}

sspcg_status sspcg_mlp_load(sspcg_mlp *n, const void *host_buf, int64_t bytes, sspcg_stream stream) {
  if (!n || !host_buf || bytes < kCkptBytes) return SSPCG_ERR_INVALID_ARG;
  CkptHeader h;
  const char *b = static_cast<const char *>(host_buf);
  std::memcpy(&h, b, sizeof(h));
  if (std::memcmp(h.magic, "SSPCGMLP", 8) != 0 || h.version != kCkptVersion || h.in != kIn || h.hidden != kHid ||
      h.out != kOut || h.params != kParams || h.steps < 0)
    return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const char *cur = b + sizeof(h);
  for (float *dst : {n->w, n->m, n->v}) {
    MLP_CUDA(cudaMemcpyAsync(dst, cur, sizeof(float) * kParams, cudaMemcpyHostToDevice, st));
    cur += sizeof(float) * kParams;
  }
  for (float *dst : {n->mu, n->isd}) {
    MLP_CUDA(cudaMemcpyAsync(dst, cur, sizeof(float) * kIn, cudaMemcpyHostToDevice, st));
    cur += sizeof(float) * kIn;
  }
  MLP_CUDA(cudaMemsetAsync(n->g, 0, sizeof(float) * kParams, st));
  n->t = h.steps;
  sspcg_status s = refresh_copies(n, st);
  if (s != SSPCG_OK) return s;
  MLP_CUDA(cudaStreamSynchronize(st));
  return SSPCG_OK;
}

sspcg_status sspcg_pipeline_warm_batched(sspcg_plan *plan, sspcg_mlp *n, sspcg_precond kind, const float *A,
                                         const float *B, const float *qd, const float *rd, const float *gamma,
                                         float *D, float *E, float *PD, float *PE, float *lambda, int32_t *iters,
                                         double *relres, int32_t *status, sspcg_stream stream) {
  if (!plan || !n || kind < 0 || kind > 2) return SSPCG_ERR_INVALID_ARG;  // features need block D^-1
  const host::PlanView v = host::plan_view(plan);
  if (v.nprob == 0) return SSPCG_OK;
  if (!qp_ok(v, A, B, qd, rd, gamma, PD) || !D || !lambda || !iters || !relres || !status ||
      (v.total_off > 0 && (!E || !PE)))
    return SSPCG_ERR_INVALID_ARG;
  if (!aligned16(qd) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  if (!layout_fits(v)) return SSPCG_ERR_UNSUPPORTED;
  sspcg_status s = host::build_half(plan, kind, A, B, qd, rd, D, E, PD, PE, status, stream);
  if (s != SSPCG_OK) return s;
  if ((s = sspcg_mlp_infer(n, plan, A, B, qd, rd, gamma, PD, lambda, stream)) != SSPCG_OK) return s;
  return host::solve_half(plan, A, B, qd, rd, gamma, PD, PE, lambda, iters, relres, status, 2, stream);
}

}  // extern "C"
