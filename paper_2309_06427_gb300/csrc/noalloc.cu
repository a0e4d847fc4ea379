// Batched PCG solve that allocates nothing: for callers that cannot call
// cudaMalloc once they run.  Examples are a model-predictive control loop on
// a real-time thread, where cudaMalloc may synchronise the device and take
// unbounded time, and a host application whose own allocator owns all device
// memory.  Its scratch (problem descriptors, work list, work-queue counters)
// lives in a file-scope __device__ array of fixed size instead of a plan.
//
// The call copies nothing from host memory with cudaMemcpy: the problem
// shapes and the work order travel as the parameter block of one set-up
// kernel (the driver copies kernel parameters when it records the launch),
// which computes the packed offsets, writes the descriptors and work list
// into the scratch array and clears the queue counters and the statuses.
// So the call never waits for the GPU, and it uses no host heap either.
#include <algorithm>
#include <atomic>
#include <cstring>

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
constexpr int kMaxProb = SSPCG_NOALLOC_MAX_PROBLEMS;

struct NoAllocScratch {
  ProbDesc desc[kMaxProb];
  int32_t work[kMaxProb];
  int32_t counters[kNoAllocCounters];
};

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Parameter block of the set-up kernel (about 24 KB, within the 32,764-byte
// kernel-parameter limit): shapes of the batch and its work order.
struct NoAllocShapes {
  int32_t nprob;
  int16_t N[kMaxProb];     // N <= SSPCG_MAX_N = 4096
  uint8_t nx[kMaxProb];    // nx, nu <= 28
  uint8_t nu[kMaxProb];
  int16_t work[kMaxProb];  // problem indices, grouped by nx, each group largest N first
};
static_assert(sizeof(NoAllocShapes) <= 32000, "set-up parameters exceed the kernel-parameter limit");

constexpr int kSetupThreads = 1024;
constexpr int kPerThread = kMaxProb / kSetupThreads;
static_assert(kMaxProb % kSetupThreads == 0, "problems per set-up thread");

// Exclusive prefix sum over the CTA (in thread order) of one value per thread.
__device__ int64_t cta_exclusive_scan(int64_t v, int64_t *wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = wsum[lane];  // kSetupThreads / 32 == 32 warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const int64_t base = wid > 0 ? wsum[wid - 1] : 0;
  __syncthreads();  // wsum is reused by the next scan
  return base + x - v;
}

// Descriptors with the packed layout of sspcg_plan_offsets (problem i of each
// array kind starts at the sum of the sizes of problems 0..i-1, each rounded
// up to 4 elements), the work list, zeroed counters and statuses.
__global__ void __launch_bounds__(kSetupThreads) noalloc_setup_kernel(const __grid_constant__ NoAllocShapes s,
                                                                      NoAllocScratch *scr, int32_t *status) {
  __shared__ int64_t wsum[32];
  const int t = threadIdx.x;
  int64_t off[7];
  for (int k = 0; k < 7; ++k) {
    int64_t local = 0;
    for (int q = 0; q < kPerThread; ++q) {
      const int i = t * kPerThread + q;
      if (i >= s.nprob) break;
      const int64_t Ni = s.N[i], n = Ni + 1, m = s.nx[i], u = s.nu[i];
      const int64_t sz[7] = {Ni * m * m, Ni * m * u, n * m, Ni * u, n * m * m, Ni * m * m, n * m};
      local += round_up(sz[k], 4);
    }
    off[k] = cta_exclusive_scan(local, wsum);
  }
  for (int q = 0; q < kPerThread; ++q) {
    const int i = t * kPerThread + q;
    if (i >= s.nprob) break;
    const int64_t Ni = s.N[i], n = Ni + 1, m = s.nx[i], u = s.nu[i];
    const int64_t sz[7] = {Ni * m * m, Ni * m * u, n * m, Ni * u, n * m * m, Ni * m * m, n * m};
    ProbDesc d;
    d.N = (int32_t)Ni; d.nx = (int32_t)m; d.nu = (int32_t)u; d.id = i;
    d.oA = off[SSPCG_ARRAY_A]; d.oB = off[SSPCG_ARRAY_B]; d.oq = off[SSPCG_ARRAY_QD]; d.orr = off[SSPCG_ARRAY_RD];
    d.odiag = off[SSPCG_ARRAY_DIAG]; d.ooff = off[SSPCG_ARRAY_OFF]; d.ovec = off[SSPCG_ARRAY_VEC];
    scr->desc[i] = d;
    scr->work[i] = s.work[i];
    status[i] = 0;
    for (int k = 0; k < 7; ++k) off[k] += round_up(sz[k], 4);
  }
  if (t < kNoAllocCounters) scr->counters[t] = 0;
}

constexpr int kMaxDevices = 64;
std::atomic<NoAllocScratch *> g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current.  Two threads that make their
// first call on one device at the same time both look it up and store the
// same value.
sspcg_status scratch_address(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return host::cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return SSPCG_ERR_UNSUPPORTED;
  NoAllocScratch *p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return host::cuda_error(e);
    p = static_cast<NoAllocScratch *>(ptr);
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return SSPCG_OK;
}

}  // namespace

extern "C" sspcg_status sspcg_solve_qp_batched_noalloc(int32_t nprob, const int32_t *N, const int32_t *nx,
                                                       const int32_t *nu, const float *A, const float *B,
                                                       const float *qd, const float *rd, const float *PD,
                                                       const float *PE, const float *gamma, float *lambda,
                                                       const sspcg_options *opts, int32_t *iters, double *relres,
                                                       int32_t *status, sspcg_stream stream) {
  if (nprob < 0 || nprob > kMaxProb) return SSPCG_ERR_INVALID_ARG;
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

  // Shapes and work order (grouped by nx, each group largest N first, ties by index) in the set-up
  // kernel's parameter block; per group the launch shape.  Fixed-size storage only.
  NoAllocShapes s;
  s.nprob = nprob;
  struct Group {
    int32_t count = 0, first = 0;
    int64_t rows = 0, smem = 0;
  } groups[kMaxNx + 1];
  for (int32_t i = 0; i < nprob; ++i) {
    s.N[i] = (int16_t)N[i];
    s.nx[i] = (uint8_t)nx[i];
    s.nu[i] = (uint8_t)nu[i];
    int K = 0;
    int64_t bytes = 0;
    if (!host::fit(kOpQp, opts->schedule, N[i], nx[i], nu[i], false, opts->poly_degree, opts->cg_variant, &K,
                   &bytes))
      return SSPCG_ERR_UNSUPPORTED;
    Group &g = groups[nx[i]];
    ++g.count;
    g.rows = std::max<int64_t>(g.rows, (int64_t)(N[i] + 1) * nx[i]);
    g.smem = std::max<int64_t>(g.smem, bytes);
  }
  int32_t pos = 0;
  for (int m = 1; m <= kMaxNx; ++m) {
    groups[m].first = pos;
    pos += groups[m].count;
  }
  {
    int32_t fill[kMaxNx + 1];
    for (int m = 0; m <= kMaxNx; ++m) fill[m] = groups[m].first;
    for (int32_t i = 0; i < nprob; ++i) s.work[fill[nx[i]]++] = (int16_t)i;
    for (int m = 1; m <= kMaxNx; ++m) {
      int16_t *w = s.work + groups[m].first;
      std::sort(w, w + groups[m].count, [&](int16_t x, int16_t y) { return N[x] != N[y] ? N[x] > N[y] : x < y; });
    }
  }

  NoAllocScratch *scr = nullptr;
  sspcg_status st_ = scratch_address(&scr);
  if (st_ != SSPCG_OK) return st_;
  cudaStream_t st = (cudaStream_t)stream;
  // stream-ordered after any earlier call on this stream; calls that overlap on the GPU race
  noalloc_setup_kernel<<<1, kSetupThreads, 0, st>>>(s, scr, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return host::cuda_error(e);

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
  int counter = 0;
  for (int m = 1; m <= kMaxNx; ++m) {
    const Group &g = groups[m];
    if (g.count == 0) continue;
    const int block = opts->block_threads > 0 ? opts->block_threads : host::block_for_rows(g.rows);
    const int by_smem = (int)std::max<int64_t>(1, (228 * 1024) / (g.smem + 2048));
    const int by_thr = std::max(1, 2048 / block);
    const int grid = (int)std::min<int64_t>(g.count, (int64_t)std::min(by_smem, by_thr) * host::sms());
    PcgArgs ga = a;
    ga.work = scr->work + g.first;
    ga.nwork = g.count;
    ga.counter = scr->counters + counter++;
    e = launch_pcg(m, kOpQp, host::reduction_mode(opts->reduction), false, ga, grid, block, (size_t)g.smem, st);
    if (e != cudaSuccess) return host::cuda_error(e);
  }
  return SSPCG_OK;
}
