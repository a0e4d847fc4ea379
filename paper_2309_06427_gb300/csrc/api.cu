// C ABI of sspcg: argument validation, batch plans, schedules and launches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/sspcg.h"
#include "common.cuh"
#include "kernels.h"

using namespace sspcg;

namespace {

thread_local char g_cuda_err[256] = "no error";

sspcg_status cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return SSPCG_ERR_CUDA;
}

#define SSPCG_CUDA(call)                         \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int max_smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return v;
}

// Static shared memory of the PCG kernels (reduction slots and the work index).
constexpr int kPcgStaticSmem = 4 * 32 * 8 + 16;

bool shape_ok(int N, int nx, int nu) {
  return N >= 0 && N <= SSPCG_MAX_N && nx >= 1 && nx <= SSPCG_MAX_NX && nu >= 0 && nu <= SSPCG_MAX_NX;
}

ProbDesc single_desc(int N, int nx, int nu) {
  ProbDesc d{};
  d.N = N; d.nx = nx; d.nu = nu;
  return d;
}

int red_mode(int32_t r) {
  if (r == SSPCG_REDUCE_F32) return kRedF32;
  if (r == SSPCG_REDUCE_F64) return kRedF64;
  return kRedDf;
}

int64_t pcg_smem_bytes(int op, bool res, int N, int nx, int nu) {
  return pcg_layout(op, res, N, nx, nu).total * (int64_t)sizeof(float);
}

int64_t smem_budget() { return (int64_t)max_smem_optin() - kPcgStaticSmem; }  // bytes of dynamic smem

// Threads per CTA for a problem with R rows: about two rows per thread.
int auto_block(int64_t rows) {
  int64_t t = round_up(cdiv(rows, 2), 32);
  return (int)std::min<int64_t>(256, std::max<int64_t>(64, t));
}

// Choose residency for a problem; returns false when even the streaming
// layout does not fit.
bool choose_resident(int op, int sched, int N, int nx, int nu, bool *resident) {
  const int64_t budget = smem_budget();
  const bool fits_res = pcg_smem_bytes(op, true, N, nx, nu) <= budget;
  const bool fits_str = pcg_smem_bytes(op, false, N, nx, nu) <= budget;
  if (!fits_str) return false;
  *resident = (sched != SSPCG_SCHED_STREAM) && fits_res;
  return true;
}

sspcg_status validate_opts(const sspcg_options *o) {
  if (!o) return SSPCG_ERR_INVALID_ARG;
  if (!(o->tol >= 0.0)) return SSPCG_ERR_INVALID_ARG;
  if (o->warm_start < 0 || o->warm_start > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->reduction < 0 || o->reduction > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->schedule < 0 || o->schedule > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->block_threads != 0 && (o->block_threads < 32 || o->block_threads > 512 || o->block_threads % 32))
    return SSPCG_ERR_INVALID_ARG;
  return SSPCG_OK;
}

}  // namespace

namespace sspcg {
// Largest dynamic shared memory of a PCG launch (opt-in limit minus the static part).
int pcg_max_smem_bytes() { return max_smem_optin() - kPcgStaticSmem; }
}  // namespace sspcg

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct PcgGroup {
  int nx = 0;
  bool resident = false;
  int block = 0;
  int grid = 0;
  size_t smem = 0;
  int32_t *d_work = nullptr;  // slice of the plan's work array
  int32_t nwork = 0;
  int counter_index = 0;
};

struct sspcg_plan {
  int32_t nprob = 0;
  sspcg_options opts{};
  std::vector<ProbDesc> hdesc;
  std::vector<int64_t> offsets[SSPCG_NUM_ARRAYS];
  int64_t sizes[SSPCG_NUM_ARRAYS] = {};
  ProbDesc *d_desc = nullptr;
  int64_t *d_knot_start = nullptr, *d_off_start = nullptr;
  int64_t total_knots = 0, total_off = 0;
  int32_t *d_work = nullptr;      // 2 * nprob: QP-form groups then block-form groups
  int32_t *d_counters = nullptr;  // one per group
  std::vector<PcgGroup> groups[2];  // [op]
  int ngroups_total = 0;
  // side streams for concurrent group launches
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  // plan-owned device buffers of the host pipeline
  float *hbuf = nullptr;
  int64_t hbuf_floats = 0;
  int32_t *hint = nullptr;
  double *hdbl = nullptr;
};

namespace {

void plan_free(sspcg_plan *p) {
  if (!p) return;
  cudaFree(p->d_desc);
  cudaFree(p->d_knot_start);
  cudaFree(p->d_off_start);
  cudaFree(p->d_work);
  cudaFree(p->d_counters);
  cudaFree(p->hbuf);
  cudaFree(p->hint);
  cudaFree(p->hdbl);
  for (auto s : p->side) cudaStreamDestroy(s);
  for (auto e : p->ev) cudaEventDestroy(e);
  delete p;
}

// Build the PCG launch groups of one operator form: problems grouped by
// (nx, residency), each group's work list ordered largest first.
sspcg_status plan_groups(sspcg_plan *p, int op, std::vector<int32_t> &work_host, int32_t base) {
  std::vector<std::vector<int32_t>> buckets(2 * (kMaxNx + 1));
  for (int32_t i = 0; i < p->nprob; ++i) {
    const ProbDesc &d = p->hdesc[i];
    bool res = false;
    if (!choose_resident(op, p->opts.schedule, d.N, d.nx, d.nu, &res)) return SSPCG_ERR_UNSUPPORTED;
    buckets[2 * d.nx + (res ? 1 : 0)].push_back(i);
  }
  int32_t pos = base;
  for (int nx = 1; nx <= kMaxNx; ++nx) {
    for (int r = 0; r < 2; ++r) {
      auto &b = buckets[2 * nx + r];
      if (b.empty()) continue;
      std::stable_sort(b.begin(), b.end(), [&](int32_t x, int32_t y) {
        return p->hdesc[x].N > p->hdesc[y].N;  // same nx: cost grows with N
      });
      PcgGroup g;
      g.nx = nx;
      g.resident = r == 1;
      int64_t maxrows = 0, maxsmem = 0;
      for (int32_t i : b) {
        const ProbDesc &d = p->hdesc[i];
        maxrows = std::max<int64_t>(maxrows, (int64_t)(d.N + 1) * d.nx);
        maxsmem = std::max<int64_t>(maxsmem, pcg_smem_bytes(op, g.resident, d.N, d.nx, d.nu));
      }
      g.block = p->opts.block_threads > 0 ? p->opts.block_threads : auto_block(maxrows);
      g.smem = (size_t)maxsmem;
      const int64_t per_sm_smem = 228 * 1024;
      int by_smem = (int)std::max<int64_t>(1, per_sm_smem / (maxsmem + kPcgStaticSmem + 1024));
      int by_thr = std::max(1, 2048 / g.block);
      int per_sm = std::min(by_smem, by_thr);
      g.grid = (int)std::min<int64_t>((int64_t)b.size(), (int64_t)per_sm * device_sms());
      g.nwork = (int32_t)b.size();
      g.d_work = p->d_work + pos;
      g.counter_index = p->ngroups_total++;
      for (int32_t i : b) work_host[pos++] = i;
      p->groups[op].push_back(g);
    }
  }
  return SSPCG_OK;
}

sspcg_status launch_groups(sspcg_plan *p, int op, const PcgArgs &base, cudaStream_t st) {
  auto &groups = p->groups[op];
  if (groups.empty()) return SSPCG_OK;
  SSPCG_CUDA(cudaMemsetAsync(p->d_counters, 0, sizeof(int32_t) * p->ngroups_total, st));
  const size_t ng = groups.size();
  // fork: side streams wait for the main stream
  if (ng > 1) {
    SSPCG_CUDA(cudaEventRecord(p->ev[0], st));
    for (size_t i = 1; i < ng; ++i) SSPCG_CUDA(cudaStreamWaitEvent(p->side[i - 1], p->ev[0], 0));
  }
  for (size_t i = 0; i < ng; ++i) {
    const PcgGroup &g = groups[i];
    PcgArgs a = base;
    a.work = g.d_work;
    a.nwork = g.nwork;
    a.counter = p->d_counters + g.counter_index;
    cudaStream_t s = i == 0 ? st : p->side[i - 1];
    SSPCG_CUDA(launch_pcg(g.nx, op, red_mode(p->opts.reduction), g.resident, a, g.grid, g.block, g.smem, s));
  }
  // join
  for (size_t i = 1; i < ng; ++i) {
    SSPCG_CUDA(cudaEventRecord(p->ev[i], p->side[i - 1]));
    SSPCG_CUDA(cudaStreamWaitEvent(st, p->ev[i], 0));
  }
  return SSPCG_OK;
}

PcgArgs make_args(const sspcg_options *o) {
  PcgArgs a{};
  a.tol2 = (float)(o->tol * o->tol);
  a.max_iter = o->max_iter;
  a.warm = o->warm_start;
  return a;
}

}  // namespace

extern "C" {

const char *sspcg_last_cuda_error(void) { return g_cuda_err; }
const char *sspcg_version(void) { return "sspcg 0.1 (sm_103a)"; }

sspcg_status sspcg_build_schur(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                               const float *rd, float *D, float *E, sspcg_stream stream) {
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!qd || !D || (N > 0 && (!A || !rd || !E || (nu > 0 && !B)))) return SSPCG_ERR_INVALID_ARG;
  ProbSet ps{nullptr, single_desc(N, nx, nu), 1};
  SSPCG_CUDA(launch_schur_build(ps, nullptr, N + 1, A, B, qd, rd, D, E, (cudaStream_t)stream, device_sms()));
  return SSPCG_OK;
}

sspcg_status sspcg_build_precond(int32_t N, int32_t nx, sspcg_precond kind, const float *D, const float *E,
                                 float *PD, float *PE, int32_t *status, sspcg_stream stream) {
  if (!shape_ok(N, nx, 0) || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (!D || !PD || !status || (N > 0 && (!E || !PE))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ProbSet ps{nullptr, single_desc(N, nx, 0), 1};
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  SSPCG_CUDA(launch_precond_build(ps, nullptr, N + 1, nullptr, N, (int)kind, D, E, PD, PE, status, st, device_sms(),
                                  (int64_t)N * nx * nx));
  return SSPCG_OK;
}

static sspcg_status solve_single(int op, int32_t N, int32_t nx, int32_t nu, const float *A, const float *B,
                                 const float *qd, const float *rd, const float *D, const float *E, const float *PD,
                                 const float *PE, const float *gamma, float *lambda, const sspcg_options *opts,
                                 int32_t *iters, double *relres, int32_t *status, sspcg_stream stream) {
  if (validate_opts(opts) != SSPCG_OK) return SSPCG_ERR_INVALID_ARG;
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!PD || !gamma || !lambda || !iters || !relres || !status || (N > 0 && !PE)) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpQp && (!qd || (N > 0 && (!A || !rd || (nu > 0 && !B))))) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpBlock && (!D || (N > 0 && !E))) return SSPCG_ERR_INVALID_ARG;
  bool res = false;
  if (!choose_resident(op, opts->schedule, N, nx, nu, &res)) return SSPCG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  PcgArgs a = make_args(opts);
  a.ps = ProbSet{nullptr, single_desc(N, nx, nu), 1};
  a.work = nullptr; a.nwork = 1; a.counter = nullptr;
  a.A = A; a.B = B; a.qd = qd; a.rd = rd; a.D = D; a.E = E; a.PD = PD; a.PE = PE;
  a.gamma = gamma; a.lambda = lambda; a.iters = iters; a.relres = relres; a.status = status;
  const int block = opts->block_threads > 0 ? opts->block_threads : auto_block((int64_t)(N + 1) * nx);
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  SSPCG_CUDA(launch_pcg(nx, op, red_mode(opts->reduction), res, a, 1, block,
                        (size_t)pcg_smem_bytes(op, res, N, nx, nu), st));
  return SSPCG_OK;
}

sspcg_status sspcg_solve(int32_t N, int32_t nx, const float *D, const float *E, const float *PD, const float *PE,
                         const float *gamma, float *lambda, const sspcg_options *opts, int32_t *iters,
                         double *relres, int32_t *status, sspcg_stream stream) {
  return solve_single(kOpBlock, N, nx, 0, nullptr, nullptr, nullptr, nullptr, D, E, PD, PE, gamma, lambda, opts,
                      iters, relres, status, stream);
}

sspcg_status sspcg_solve_qp(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                            const float *rd, const float *PD, const float *PE, const float *gamma, float *lambda,
                            const sspcg_options *opts, int32_t *iters, double *relres, int32_t *status,
                            sspcg_stream stream) {
  return solve_single(kOpQp, N, nx, nu, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, opts, iters, relres,
                      status, stream);
}

sspcg_status sspcg_residual_qp(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                               const float *rd, const float *gamma, const float *lambda, double *relres_true,
                               sspcg_stream stream) {
  if (!shape_ok(N, nx, nu) || !qd || !gamma || !lambda || !relres_true) return SSPCG_ERR_INVALID_ARG;
  if (N > 0 && (!A || !rd || (nu > 0 && !B))) return SSPCG_ERR_INVALID_ARG;
  ProbSet ps{nullptr, single_desc(N, nx, nu), 1};
  SSPCG_CUDA(launch_residual_qp(ps, A, B, qd, rd, gamma, lambda, relres_true, (cudaStream_t)stream));
  return SSPCG_OK;
}

// ---------------------------------------------------------------------------
// Batched
// ---------------------------------------------------------------------------
sspcg_status sspcg_plan_create(sspcg_plan **plan, int32_t nprob, const int32_t *N, const int32_t *nx,
                               const int32_t *nu, const sspcg_options *opts) {
  if (!plan || nprob < 0 || (nprob > 0 && (!N || !nx || !nu))) return SSPCG_ERR_INVALID_ARG;
  if (validate_opts(opts) != SSPCG_OK) return SSPCG_ERR_INVALID_ARG;
  *plan = nullptr;
  for (int32_t i = 0; i < nprob; ++i)
    if (!shape_ok(N[i], nx[i], nu[i])) return SSPCG_ERR_INVALID_ARG;
  sspcg_plan *p = new sspcg_plan();
  p->nprob = nprob;
  p->opts = *opts;
  p->hdesc.resize(nprob);
  for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) p->offsets[k].resize(nprob);
  std::vector<int64_t> knot_start(nprob + 1, 0), off_start(nprob + 1, 0);
  int64_t cur[SSPCG_NUM_ARRAYS] = {};
  for (int32_t i = 0; i < nprob; ++i) {
    const int64_t n = N[i] + 1, m = nx[i], u = nu[i], Ni = N[i];
    const int64_t sz[SSPCG_NUM_ARRAYS] = {Ni * m * m, Ni * m * u, n * m, Ni * u, n * m * m, Ni * m * m, n * m};
    for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) {
      p->offsets[k][i] = cur[k];
      cur[k] += round_up(sz[k], 4);  // 16-byte aligned problem starts
    }
    ProbDesc &d = p->hdesc[i];
    d.N = N[i]; d.nx = nx[i]; d.nu = nu[i];
    d.oA = p->offsets[SSPCG_ARRAY_A][i];
    d.oB = p->offsets[SSPCG_ARRAY_B][i];
    d.oq = p->offsets[SSPCG_ARRAY_QD][i];
    d.orr = p->offsets[SSPCG_ARRAY_RD][i];
    d.odiag = p->offsets[SSPCG_ARRAY_DIAG][i];
    d.ooff = p->offsets[SSPCG_ARRAY_OFF][i];
    d.ovec = p->offsets[SSPCG_ARRAY_VEC][i];
    knot_start[i + 1] = knot_start[i] + n;
    off_start[i + 1] = off_start[i] + Ni;
  }
  for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) p->sizes[k] = cur[k];
  p->total_knots = knot_start[nprob];
  p->total_off = off_start[nprob];
  auto fail = [&](sspcg_status s) { plan_free(p); return s; };
  if (nprob > 0) {
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_desc, sizeof(ProbDesc) * nprob)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&p->d_knot_start, sizeof(int64_t) * (nprob + 1))) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&p->d_off_start, sizeof(int64_t) * (nprob + 1))) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&p->d_work, sizeof(int32_t) * 2 * nprob)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMemcpy(p->d_desc, p->hdesc.data(), sizeof(ProbDesc) * nprob, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e));
    if ((e = cudaMemcpy(p->d_knot_start, knot_start.data(), sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return fail(cuda_fail(e));
    if ((e = cudaMemcpy(p->d_off_start, off_start.data(), sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return fail(cuda_fail(e));
    std::vector<int32_t> work(2 * nprob);
    sspcg_status s = plan_groups(p, kOpQp, work, 0);
    if (s != SSPCG_OK) return fail(s);
    s = plan_groups(p, kOpBlock, work, nprob);
    if (s != SSPCG_OK) return fail(s);
    if ((e = cudaMemcpy(p->d_work, work.data(), sizeof(int32_t) * 2 * nprob, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e));
    if ((e = cudaMalloc(&p->d_counters, sizeof(int32_t) * std::max(1, p->ngroups_total))) != cudaSuccess)
      return fail(cuda_fail(e));
    const size_t nside = std::max(p->groups[0].size(), p->groups[1].size());
    p->ev.resize(nside + 1);
    for (auto &ev : p->ev)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(cuda_fail(e));
    p->side.resize(nside);
    for (auto &s2 : p->side)
      if ((e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess) return fail(cuda_fail(e));
  }
  *plan = p;
  return SSPCG_OK;
}

sspcg_status sspcg_plan_destroy(sspcg_plan *plan) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  plan_free(plan);
  return SSPCG_OK;
}

sspcg_status sspcg_plan_sizes(const sspcg_plan *plan, int64_t *out) {
  if (!plan || !out) return SSPCG_ERR_INVALID_ARG;
  for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) out[k] = plan->sizes[k];
  return SSPCG_OK;
}

sspcg_status sspcg_plan_offsets(const sspcg_plan *plan, sspcg_array kind, int64_t *out) {
  if (!plan || !out || kind < 0 || kind >= SSPCG_NUM_ARRAYS) return SSPCG_ERR_INVALID_ARG;
  std::memcpy(out, plan->offsets[kind].data(), sizeof(int64_t) * plan->nprob);
  return SSPCG_OK;
}

sspcg_status sspcg_plan_stats(const sspcg_plan *plan, int64_t *out) {
  if (!plan || !out) return SSPCG_ERR_INVALID_ARG;
  for (int op = 0; op < 2; ++op) {
    int64_t res = 0, str = 0;
    for (const PcgGroup &g : plan->groups[op]) (g.resident ? res : str) += g.nwork;
    const int slot = op == kOpQp ? 0 : 3;
    out[slot] = (int64_t)plan->groups[op].size();
    out[slot + 1] = res;
    out[slot + 2] = str;
  }
  return SSPCG_OK;
}

static ProbSet plan_set(const sspcg_plan *p) { return ProbSet{p->d_desc, ProbDesc{}, p->nprob}; }

sspcg_status sspcg_build_schur_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                       const float *rd, float *D, float *E, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!qd || !D || !aligned16(qd) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  if (plan->total_off > 0 && (!A || !rd || !E || !B)) return SSPCG_ERR_INVALID_ARG;
  SSPCG_CUDA(launch_schur_build(plan_set(plan), plan->d_knot_start, plan->total_knots, A, B, qd, rd, D, E,
                                (cudaStream_t)stream, device_sms()));
  return SSPCG_OK;
}

sspcg_status sspcg_build_precond_batched(sspcg_plan *plan, sspcg_precond kind, const float *D, const float *E,
                                         float *PD, float *PE, int32_t *status, sspcg_stream stream) {
  if (!plan || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!D || !PD || !status || (plan->total_off > 0 && (!E || !PE))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  SSPCG_CUDA(launch_precond_build(plan_set(plan), plan->d_knot_start, plan->total_knots, plan->d_off_start,
                                  plan->total_off, (int)kind, D, E, PD, PE, status, st, device_sms(),
                                  plan->sizes[SSPCG_ARRAY_OFF]));
  return SSPCG_OK;
}

static sspcg_status solve_batched(sspcg_plan *plan, int op, const float *A, const float *B, const float *qd,
                                  const float *rd, const float *D, const float *E, const float *PD, const float *PE,
                                  const float *gamma, float *lambda, int32_t *iters, double *relres,
                                  int32_t *status, sspcg_stream stream, bool status_in) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!PD || !gamma || !lambda || !iters || !relres || !status) return SSPCG_ERR_INVALID_ARG;
  if (plan->total_off > 0 && !PE) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpQp && (!qd || (plan->total_off > 0 && (!A || !rd || !B)))) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpBlock && (!D || (plan->total_off > 0 && !E))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!status_in) SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  PcgArgs a = make_args(&plan->opts);
  a.ps = plan_set(plan);
  a.A = A; a.B = B; a.qd = qd; a.rd = rd; a.D = D; a.E = E; a.PD = PD; a.PE = PE;
  a.gamma = gamma; a.lambda = lambda; a.iters = iters; a.relres = relres; a.status = status;
  return launch_groups(plan, op, a, st);
}

sspcg_status sspcg_solve_batched(sspcg_plan *plan, const float *D, const float *E, const float *PD,
                                 const float *PE, const float *gamma, float *lambda, int32_t *iters,
                                 double *relres, int32_t *status, sspcg_stream stream) {
  return solve_batched(plan, kOpBlock, nullptr, nullptr, nullptr, nullptr, D, E, PD, PE, gamma, lambda, iters,
                       relres, status, stream, false);
}

sspcg_status sspcg_solve_qp_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                    const float *rd, const float *PD, const float *PE, const float *gamma,
                                    float *lambda, int32_t *iters, double *relres, int32_t *status,
                                    sspcg_stream stream) {
  return solve_batched(plan, kOpQp, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters, relres, status,
                       stream, false);
}

sspcg_status sspcg_residual_qp_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                       const float *rd, const float *gamma, const float *lambda,
                                       double *relres_true, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!qd || !gamma || !lambda || !relres_true || (plan->total_off > 0 && (!A || !B || !rd)))
    return SSPCG_ERR_INVALID_ARG;
  SSPCG_CUDA(launch_residual_qp(plan_set(plan), A, B, qd, rd, gamma, lambda, relres_true, (cudaStream_t)stream));
  return SSPCG_OK;
}

sspcg_status sspcg_pipeline_batched(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                    const float *qd, const float *rd, const float *gamma, float *D, float *E,
                                    float *PD, float *PE, float *lambda, int32_t *iters, double *relres,
                                    int32_t *status, sspcg_stream stream) {
  sspcg_status s = sspcg_build_schur_batched(plan, A, B, qd, rd, D, E, stream);
  if (s != SSPCG_OK) return s;
  s = sspcg_build_precond_batched(plan, kind, D, E, PD, PE, status, stream);
  if (s != SSPCG_OK) return s;
  return solve_batched(plan, kOpQp, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters, relres, status,
                       stream, true);
}

sspcg_status sspcg_pipeline_host(sspcg_plan *plan, sspcg_precond kind, const float *A_host, const float *B_host,
                                 const float *qd_host, const float *rd_host, const float *gamma_host,
                                 float *lambda_host, int32_t *iters_host, double *relres_host, int32_t *status_host,
                                 sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!qd_host || !gamma_host || !lambda_host || !iters_host || !relres_host || !status_host)
    return SSPCG_ERR_INVALID_ARG;
  const int64_t *sz = plan->sizes;
  const int64_t need = sz[SSPCG_ARRAY_A] + sz[SSPCG_ARRAY_B] + sz[SSPCG_ARRAY_QD] + sz[SSPCG_ARRAY_RD] +
                       2 * sz[SSPCG_ARRAY_DIAG] + 2 * sz[SSPCG_ARRAY_OFF] + 2 * sz[SSPCG_ARRAY_VEC] + 64;
  if (plan->hbuf_floats < need) {
    cudaFree(plan->hbuf);
    cudaFree(plan->hint);
    cudaFree(plan->hdbl);
    plan->hbuf = nullptr; plan->hint = nullptr; plan->hdbl = nullptr; plan->hbuf_floats = 0;
    SSPCG_CUDA(cudaMalloc(&plan->hbuf, sizeof(float) * need));
    SSPCG_CUDA(cudaMalloc(&plan->hint, sizeof(int32_t) * 2 * plan->nprob));
    SSPCG_CUDA(cudaMalloc(&plan->hdbl, sizeof(double) * plan->nprob));
    plan->hbuf_floats = need;
  }
  float *cur = plan->hbuf;
  auto take = [&](int64_t n) { float *r = cur; cur += round_up(std::max<int64_t>(n, 4), 4); return r; };
  float *A = take(sz[SSPCG_ARRAY_A]), *B = take(sz[SSPCG_ARRAY_B]), *qd = take(sz[SSPCG_ARRAY_QD]);
  float *rd = take(sz[SSPCG_ARRAY_RD]), *D = take(sz[SSPCG_ARRAY_DIAG]), *E = take(sz[SSPCG_ARRAY_OFF]);
  float *PD = take(sz[SSPCG_ARRAY_DIAG]), *PE = take(sz[SSPCG_ARRAY_OFF]);
  float *g = take(sz[SSPCG_ARRAY_VEC]), *lam = take(sz[SSPCG_ARRAY_VEC]);
  int32_t *iters = plan->hint, *status = plan->hint + plan->nprob;
  double *relres = plan->hdbl;
  cudaStream_t st = (cudaStream_t)stream;
  auto h2d = [&](float *dst, const float *src, int64_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice, st);
  };
  cudaError_t e;
  if ((e = h2d(A, A_host, sz[SSPCG_ARRAY_A])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(B, B_host, sz[SSPCG_ARRAY_B])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(qd, qd_host, sz[SSPCG_ARRAY_QD])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(rd, rd_host, sz[SSPCG_ARRAY_RD])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(g, gamma_host, sz[SSPCG_ARRAY_VEC])) != cudaSuccess) return cuda_fail(e);
  if (plan->opts.warm_start && (e = h2d(lam, lambda_host, sz[SSPCG_ARRAY_VEC])) != cudaSuccess) return cuda_fail(e);
  sspcg_status s = sspcg_pipeline_batched(plan, kind, A, B, qd, rd, g, D, E, PD, PE, lam, iters, relres, status,
                                          stream);
  if (s != SSPCG_OK) return s;
  SSPCG_CUDA(cudaMemcpyAsync(lambda_host, lam, sizeof(float) * sz[SSPCG_ARRAY_VEC], cudaMemcpyDeviceToHost, st));
  SSPCG_CUDA(cudaMemcpyAsync(iters_host, iters, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToHost, st));
  SSPCG_CUDA(cudaMemcpyAsync(status_host, status, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToHost, st));
  SSPCG_CUDA(cudaMemcpyAsync(relres_host, relres, sizeof(double) * plan->nprob, cudaMemcpyDeviceToHost, st));
  SSPCG_CUDA(cudaStreamSynchronize(st));
  return SSPCG_OK;
}

}  // extern "C"
