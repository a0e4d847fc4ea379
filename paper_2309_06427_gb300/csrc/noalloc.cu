// Batched PCG solve that allocates nothing: for callers that cannot call
// cudaMalloc once they run.  Examples are a model-predictive control loop on
// a real-time thread, where cudaMalloc may synchronise the device and take
// unbounded time, and a host application whose own allocator owns all device
// memory.  Its scratch (problem descriptors, work list, work-queue counters)
// lives in a file-scope __device__ array of fixed size instead of a plan.
#include <algorithm>
#include <vector>

#include "../../include/sspcg.h"
#include "common.cuh"
#include "kernels.h"

namespace sspcg {
namespace host {  // defined in api.cu
int sms();
int reduction_mode(int32_t r);
int block_for_rows(int64_t rows);
bool fit(int op, int sched, int N, int nx, int nu, bool f64, int poly, int cg, int *K, int64_t *bytes);
sspcg_status check_options(const sspcg_options *o);
bool valid_shape(int N, int nx, int nu);
sspcg_status cuda_error(cudaError_t e);
}  // namespace host
}  // namespace sspcg

using namespace sspcg;

namespace {

constexpr int kNoAllocCounters = 64;

struct NoAllocScratch {
  ProbDesc desc[SSPCG_NOALLOC_MAX_PROBLEMS];
  int32_t work[SSPCG_NOALLOC_MAX_PROBLEMS];
  int32_t counters[kNoAllocCounters];
};

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current.
sspcg_status scratch_address(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return host::cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return SSPCG_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return host::cuda_error(e);
    g_scratch_addr[dev] = static_cast<NoAllocScratch *>(ptr);
  }
  *out = g_scratch_addr[dev];
  return SSPCG_OK;
}

}  // namespace

extern "C" sspcg_status sspcg_solve_qp_batched_noalloc(int32_t nprob, const int32_t *N, const int32_t *nx,
                                                       const int32_t *nu, const float *A, const float *B,
                                                       const float *qd, const float *rd, const float *PD,
                                                       const float *PE, const float *gamma, float *lambda,
                                                       const sspcg_options *opts, int32_t *iters, double *relres,
                                                       int32_t *status, sspcg_stream stream) {
  if (nprob < 0 || nprob > SSPCG_NOALLOC_MAX_PROBLEMS) return SSPCG_ERR_INVALID_ARG;
  if (host::check_options(opts) != SSPCG_OK) return SSPCG_ERR_INVALID_ARG;
  if (nprob == 0) return SSPCG_OK;
  if (!N || !nx || !nu) return SSPCG_ERR_INVALID_ARG;
  int64_t total_off = 0;
  for (int32_t i = 0; i < nprob; ++i) {
    if (!host::valid_shape(N[i], nx[i], nu[i])) return SSPCG_ERR_INVALID_ARG;
    total_off += N[i];
  }
  if (!qd || !PD || !gamma || !lambda || !iters || !relres || !status) return SSPCG_ERR_INVALID_ARG;
  if (total_off > 0 && (!A || !B || !rd || !PE)) return SSPCG_ERR_INVALID_ARG;

  // Descriptors with the packed layout of sspcg_plan_offsets; groups by nx.
  std::vector<ProbDesc> desc(nprob);
  int64_t cur[SSPCG_NUM_ARRAYS] = {};
  std::vector<std::vector<int32_t>> by_nx(kMaxNx + 1);
  std::vector<int64_t> bytes(nprob, 0);
  for (int32_t i = 0; i < nprob; ++i) {
    const int64_t n = N[i] + 1, m = nx[i], u = nu[i], Ni = N[i];
    const int64_t sz[SSPCG_NUM_ARRAYS] = {Ni * m * m, Ni * m * u, n * m, Ni * u, n * m * m, Ni * m * m, n * m};
    int64_t off[SSPCG_NUM_ARRAYS];
    for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) {
      off[k] = cur[k];
      cur[k] += round_up(sz[k], 4);
    }
    ProbDesc &d = desc[i];
    d.N = N[i]; d.nx = nx[i]; d.nu = nu[i]; d.id = i;
    d.oA = off[SSPCG_ARRAY_A]; d.oB = off[SSPCG_ARRAY_B]; d.oq = off[SSPCG_ARRAY_QD]; d.orr = off[SSPCG_ARRAY_RD];
    d.odiag = off[SSPCG_ARRAY_DIAG]; d.ooff = off[SSPCG_ARRAY_OFF]; d.ovec = off[SSPCG_ARRAY_VEC];
    int K = 0;
    if (!host::fit(kOpQp, opts->schedule, d.N, d.nx, d.nu, false, opts->poly_degree, opts->cg_variant, &K, &bytes[i]))
      return SSPCG_ERR_UNSUPPORTED;
    by_nx[d.nx].push_back(i);
  }
  struct Group {
    int nx, block, grid, counter;
    int32_t first, count;
    size_t smem;
  };
  std::vector<Group> groups;
  std::vector<int32_t> work;
  work.reserve(nprob);
  for (int m = 1; m <= kMaxNx; ++m) {
    auto &b = by_nx[m];
    if (b.empty()) continue;
    std::stable_sort(b.begin(), b.end(), [&](int32_t x, int32_t y) { return desc[x].N > desc[y].N; });
    Group g;
    g.nx = m;
    g.first = (int32_t)work.size();
    g.count = (int32_t)b.size();
    g.counter = (int)groups.size();
    int64_t rows = 0, smem = 0;
    for (int32_t i : b) {
      rows = std::max<int64_t>(rows, (int64_t)(desc[i].N + 1) * m);
      smem = std::max<int64_t>(smem, bytes[i]);
      work.push_back(i);
    }
    g.block = opts->block_threads > 0 ? opts->block_threads : host::block_for_rows(rows);
    g.smem = (size_t)smem;
    const int by_smem = (int)std::max<int64_t>(1, (228 * 1024) / (smem + 2048));
    const int by_thr = std::max(1, 2048 / g.block);
    g.grid = (int)std::min<int64_t>(g.count, (int64_t)std::min(by_smem, by_thr) * host::sms());
    groups.push_back(g);
  }

  NoAllocScratch *scr = nullptr;
  sspcg_status s = scratch_address(&scr);
  if (s != SSPCG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  // stream-ordered after any earlier call on this stream; calls that overlap on the GPU race
  if ((e = cudaMemcpyAsync(scr->desc, desc.data(), sizeof(ProbDesc) * nprob, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return host::cuda_error(e);
  if ((e = cudaMemcpyAsync(scr->work, work.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return host::cuda_error(e);
  if ((e = cudaMemsetAsync(scr->counters, 0, sizeof(scr->counters), st)) != cudaSuccess) return host::cuda_error(e);
  if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t) * nprob, st)) != cudaSuccess) return host::cuda_error(e);

  PcgArgs a{};
  a.ps = ProbSet{scr->desc, ProbDesc{}, nprob};
  a.A = A; a.B = B; a.qd = qd; a.rd = rd; a.PD = PD; a.PE = PE;
  a.gamma = gamma; a.lambda = lambda; a.iters = iters; a.relres = relres; a.status = status;
  a.tol2 = (float)(opts->tol * opts->tol);
  a.max_iter = opts->max_iter;
  a.warm = opts->warm_start;
  a.poly = opts->poly_degree;
  a.cg = opts->cg_variant;
  a.lambda_f32 = 1;
  a.max_resident = opts->schedule == SSPCG_SCHED_STREAM ? 0 : (1 << 30);
  for (const Group &g : groups) {
    PcgArgs ga = a;
    ga.work = scr->work + g.first;
    ga.nwork = g.count;
    ga.counter = scr->counters + g.counter;
    e = launch_pcg(g.nx, kOpQp, host::reduction_mode(opts->reduction), false, ga, g.grid, g.block, g.smem, st);
    if (e != cudaSuccess) return host::cuda_error(e);
  }
  return SSPCG_OK;
}
