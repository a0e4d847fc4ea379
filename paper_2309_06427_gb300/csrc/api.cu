// C ABI of sspcg: argument validation, batch plans, schedules and launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/sspcg.h"
#include "common.cuh"
#include "host.h"
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

// Device attribute of the current device, cached per device (devices beyond 63 query every time).
int device_attr(cudaDeviceAttr what, std::atomic<int> (&cache)[64], int fallback) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&v, what, dev) != cudaSuccess || v <= 0) v = fallback;
  if (cached) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

std::atomic<int> g_sms[64], g_smem_optin[64];

int device_sms() { return device_attr(cudaDevAttrMultiProcessorCount, g_sms, 1); }

int max_smem_optin() { return device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, g_smem_optin, 48 * 1024); }

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

int64_t smem_budget() { return (int64_t)max_smem_optin() - kPcgStaticSmem; }  // bytes of dynamic smem

// Threads per CTA for a problem with R rows: about two rows per thread, 64 to 512 threads.  Measured on
// uniform batches: two rows per thread beats one (fewer threads at each of the five CTA barriers of an
// iteration, more CTAs per SM); nx = 4, N = 64 (260 rows) runs 1.6x faster at 128 threads than at 288.
int auto_block(int64_t rows) {
  int64_t t = round_up((rows + 1) / 2, 32);
  return (int)std::min<int64_t>(512, std::max<int64_t>(64, t));
}

// Staged block rows K and dynamic shared memory (bytes) of a PCG problem
// under a schedule; false when even the vectors do not fit.
// cg: the options ask for single-reduction PCG, which the QP-form FP32 launches run (two more vectors).
// share: the problem's CTA gets 1/share of the dynamic shared-memory budget (share > 1 lets several CTAs of a
// partially staged group share an SM, each staging fewer block rows).
bool pcg_fit(int op, int sched, int N, int nx, int nu, bool f64, int poly, int cg, int *K, int64_t *bytes,
             int share = 1) {
  const int64_t esz = f64 ? sizeof(double) : sizeof(float);
  const int64_t budget = smem_budget() / share / esz;
  cg = (cg && op == kOpQp && !f64) ? 1 : 0;
  int k = pcg_max_resident(op, N, nx, nu, budget, poly > 0, cg);
  if (k < 0) return false;
  // A problem that does not fit whole stages its first k block rows and streams the rest.  (Streaming
  // everything wins on a uniform batch of large problems, where it has the L2 bandwidth to itself, but
  // loses on the ragged batch, where the concurrent groups share it.)
  if (sched == SSPCG_SCHED_STREAM && N > 0) k = 0;  // a single knot stays staged (see pcg_layout)
  *K = k;
  *bytes = pcg_layout(op, k, N, nx, nu, poly > 0, cg).total * esz;
  return true;
}

// Global-workspace slot (elements, a multiple of 4) of a problem whose vectors do not fit in shared memory.
int64_t gvec_slot(int op, int N, int nx, int nu, int poly, int cg) {
  return round_up(pcg_layout(op, 0, N, nx, nu, poly > 0, cg && op == kOpQp).total, 4);
}

sspcg_status validate_opts(const sspcg_options *o) {
  if (!o) return SSPCG_ERR_INVALID_ARG;
  if (!(o->tol >= 0.0)) return SSPCG_ERR_INVALID_ARG;
  if (o->warm_start < 0 || o->warm_start > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->reduction < 0 || o->reduction > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->schedule < 0 || o->schedule > 3) return SSPCG_ERR_INVALID_ARG;
  if (o->block_threads != 0 && (o->block_threads < 32 || o->block_threads > 512 || o->block_threads % 32))
    return SSPCG_ERR_INVALID_ARG;
  if (o->precision < 0 || o->precision > 2) return SSPCG_ERR_INVALID_ARG;
  if (o->poly_degree < 0 || o->poly_degree > SSPCG_MAX_POLY_DEGREE) return SSPCG_ERR_INVALID_ARG;
  if (o->cg_variant < 0 || o->cg_variant > 1) return SSPCG_ERR_INVALID_ARG;
  if (o->cg_variant == 1 && o->reduction != SSPCG_REDUCE_DF) return SSPCG_ERR_INVALID_ARG;
  return SSPCG_OK;
}

}  // namespace

namespace sspcg {
// Largest dynamic shared memory of a PCG launch (opt-in limit minus the static part).
int pcg_max_smem_bytes() { return max_smem_optin() - kPcgStaticSmem; }

// Host helpers shared with the other entry-point units.
namespace host {
int sms() { return device_sms(); }
int reduction_mode(int32_t r) { return red_mode(r); }
int block_for_rows(int64_t rows) { return auto_block(rows); }
bool fit(int op, int sched, int N, int nx, int nu, bool f64, int poly, int cg, int *K, int64_t *bytes) {
  return pcg_fit(op, sched, N, nx, nu, f64, poly, cg, K, bytes);
}
sspcg_status check_options(const sspcg_options *o) { return validate_opts(o); }
bool valid_shape(int N, int nx, int nu) { return shape_ok(N, nx, nu); }
sspcg_status cuda_error(cudaError_t e) { return cuda_fail(e); }
}  // namespace host
}  // namespace sspcg

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
// Problems with at most this many unknowns ((N+1)*nx) take the FP64 path in
// the pipeline calls under SSPCG_PRECISION_AUTO: in FP32 their CG loses the
// finite termination that the clustered spectrum of Thm. 4.2 gives in exact
// arithmetic (a few extra iterations), and at this size FP64 costs little.
constexpr int64_t kTinyUnknowns = 192;

struct PcgGroup {
  int nx = 0;
  int cls = 0;               // residency class (see plan_groups)
  bool resident = false;
  bool f64 = false;
  bool gvec = false;         // vectors in a global workspace (slot_elems per CTA from scratch_off)
  bool stream = false;       // stage no block rows (the schedule option, or the tuner's choice)
  int share = 1;             // partially staged groups: stage into 1/share of the shared memory (tuner's choice)
  int warps = 0;             // > 0: one problem per warp, this many warps per CTA (tuner's choice; see warp_ok)
  bool tuned = false;        // block and residency from the tuner (this plan's, or its cache)
  int64_t slot_elems = 0, scratch_off = 0;
  int max_grid = 0;          // global-vector groups: CTAs the workspace holds
  int block = 0;
  int grid = 0;
  size_t smem = 0;
  int32_t *d_work = nullptr;  // slice of the plan's work array
  int32_t nwork = 0;
  int counter_index = 0;
  int32_t maxN = 0;
  int64_t maxrows = 0;
  std::vector<int32_t> members;  // indices into the set's descriptors, in work-list order
  double work = 0.0;  // estimated PCG work: sum over members of (N+1)^1.5 nx (3 nx + nu)
};

// A set of problems solved by one group of PCG launches (one per nx and schedule).
struct GroupSet {
  int id = 0;  // which set of the plan (the tuning cache keeps each set's choices apart)
  int op = kOpQp;
  bool f64 = false;
  std::vector<PcgGroup> groups;
  int64_t n_resident = 0, n_stream = 0, n_gvec = 0;
  int64_t scratch_elems = 0;  // global workspace of its global-vector groups
  bool unsupported = false;   // holds problems that this set's operator form cannot solve
};

enum { kSetQpAll = 0, kSetBlockAll = 1, kSetQpMain = 2, kSetTiny = 3, kNumSets = 4 };

// Problems of one nx, for the thread-per-knot kernels.
struct NxGroup {
  int nx = 0;
  int mx = 1;  // largest nx and nu of the group
  int32_t nprob = 0;
  int64_t knots = 0, offs = 0;
  ProbDesc *d_desc = nullptr;
  int2 *d_refs = nullptr;   // (index into d_desc, block row) per knot
  int2 *d_orefs = nullptr;  // (index into d_desc, block row) per off-diagonal block
};

struct sspcg_plan {
  int32_t nprob = 0;
  int mx = 1;       // largest nx and nu of the batch
  int mx_tiny = 1;  // of its FP64 subset
  std::vector<NxGroup> nxg_all, nxg_tiny;
  sspcg_options opts{};
  std::vector<ProbDesc> hdesc;
  std::vector<int64_t> offsets[SSPCG_NUM_ARRAYS];
  int64_t sizes[SSPCG_NUM_ARRAYS] = {};
  ProbDesc *d_desc = nullptr;
  int2 *d_kref = nullptr, *d_oref = nullptr;  // (problem, block row) per knot / off-diagonal block
  int64_t total_knots = 0, total_off = 0;
  std::vector<int64_t> knot_start;      // first knot (index into d_kref) of each problem, nprob + 1 entries
  int64_t *d_knot_start = nullptr;
  // FP64 subset: descriptors whose odiag/ooff point into plan-owned FP64 blocks
  int32_t ntiny = 0;
  std::vector<ProbDesc> tdesc;
  ProbDesc *d_tdesc = nullptr;
  int2 *d_tkref = nullptr, *d_toref = nullptr;
  int64_t tknots = 0, toff = 0, t_diag = 0, t_offe = 0;
  double *D64 = nullptr, *E64 = nullptr, *PD64 = nullptr, *PE64 = nullptr;
  // global workspace of the global-vector groups (shared by the sets, which never run concurrently;
  // the pipeline's FP32 and FP64 sets take disjoint parts)
  void *d_scratch = nullptr;
  int64_t tiny_scratch_byte_off = 0;  // the FP64 set's part in the pipeline
  // PCG launch groups
  int32_t *d_work = nullptr;
  int32_t *d_counters = nullptr;
  int ngroups_total = 0;
  GroupSet sets[kNumSets];
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  // phase timing (opt-in)
  bool timing = false;
  cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};
  bool build_timed = false;
  // captured pipeline
  cudaGraphExec_t graph = nullptr;
  // plan-owned device buffers of the host pipeline
  float *hbuf = nullptr;
  int64_t hbuf_floats = 0;
  int32_t *hint = nullptr;
  double *hdbl = nullptr;
  // asynchronous host pipeline: two input/output slots, shared block buffers, copy streams
  struct AsyncSlot {
    float *buf = nullptr;  // A, B, qd, rd, gamma, lambda
    int32_t *ints = nullptr;
    double *dbl = nullptr;
    cudaEvent_t in_ready = nullptr, consumed = nullptr, computed = nullptr, out_done = nullptr;
  } aslot[2];
  float *ablocks = nullptr;  // D, E, PD, PE
  cudaStream_t h2d = nullptr, d2h = nullptr;
  int64_t acalls = 0;
  // full SPD cost blocks: Q^-1 (laid out like D), R^-1 (like the R input), R-block groups by nu
  float *qinv = nullptr, *rinv = nullptr;
  int64_t *d_roff = nullptr;
  std::vector<NxGroup> nxg_r;
  bool full_ready = false;
  // padded copies of A, B and PE for the problems whose block rows stream (QP form, FP32 sets): the PCG
  // reads their streamed rows 16 bytes at a time (launch_pad_rows)
  float *d_pad = nullptr;
  int64_t *d_pad_off = nullptr;  // per problem: offset in d_pad, or -1
  int32_t *d_pad_list = nullptr;  // the padded problems (indices into d_desc)
  int32_t npad = 0;
};

namespace {

void plan_free(sspcg_plan *p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (void *ptr : {(void *)p->d_desc, (void *)p->d_kref, (void *)p->d_oref, (void *)p->d_knot_start, (void *)p->d_tdesc,
                    (void *)p->d_tkref, (void *)p->d_toref, (void *)p->D64, (void *)p->E64,
                    (void *)p->PD64, (void *)p->PE64, (void *)p->d_work, (void *)p->d_counters, (void *)p->d_scratch, (void *)p->hbuf,
                    (void *)p->hint, (void *)p->hdbl, (void *)p->d_pad, (void *)p->d_pad_off, (void *)p->d_pad_list})
    cudaFree(ptr);
  for (auto *v : {&p->nxg_all, &p->nxg_tiny})
    for (NxGroup &g : *v) {
      cudaFree(g.d_desc);
      cudaFree(g.d_refs);
      cudaFree(g.d_orefs);
    }
  for (auto &a : p->aslot) {
    cudaFree(a.buf);
    cudaFree(a.ints);
    cudaFree(a.dbl);
    for (cudaEvent_t e : {a.in_ready, a.consumed, a.computed, a.out_done})
      if (e) cudaEventDestroy(e);
  }
  cudaFree(p->ablocks);
  cudaFree(p->qinv);
  cudaFree(p->rinv);
  cudaFree(p->d_roff);
  for (NxGroup &g : p->nxg_r) {
    cudaFree(g.d_desc);
    cudaFree(g.d_refs);
    cudaFree(g.d_orefs);
  }
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  for (auto s : p->side) cudaStreamDestroy(s);
  for (auto e : p->ev) cudaEventDestroy(e);
  for (auto e : p->tev)
    if (e) cudaEventDestroy(e);
  delete p;
}

// Tuning cache: the block size and residency the tuner picked, per (operator form, precision, reduction,
// polynomial degree, PCG variant, nx, residency class, bucket of the group's largest N).  Process-wide; plans
// created after a tuning run take its choices for groups with the same key.
struct TuneKey {
  int set, op, f64, red, poly, cg, nx, cls, nbucket;
  bool operator<(const TuneKey &o) const {
    const int a[9] = {set, op, f64, red, poly, cg, nx, cls, nbucket};
    const int b[9] = {o.set, o.op, o.f64, o.red, o.poly, o.cg, o.nx, o.cls, o.nbucket};
    return std::lexicographical_compare(a, a + 9, b, b + 9);
  }
};
struct TuneChoice {
  int block;
  bool stream;
  int share;
  int warps;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

int n_bucket(int32_t maxN) {
  int b = 0;
  while (b < 6 && maxN >= (16 << b)) ++b;  // <16, <32, <64, <128, <256, <512, >= 512
  return b;
}

TuneKey tune_key(const sspcg_plan *p, const GroupSet &set, const PcgGroup &g) {
  return TuneKey{set.id, set.op, set.f64 ? 1 : 0, set.f64 ? kRedF64 : red_mode(p->opts.reduction), p->opts.poly_degree,
                 (p->opts.cg_variant && set.op == kOpQp && !set.f64) ? 1 : 0, g.nx, g.cls, n_bucket(g.maxN)};
}

// One problem per warp exists for fully staged groups of the QP form with textbook PCG: the FP64 path, and
// FP32 with double-float sums.
bool warp_ok(const sspcg_plan *p, const GroupSet &set, const PcgGroup &g) {
  if (set.op != kOpQp || g.gvec || g.cls < 1 || g.cls > 4) return false;
  if (set.f64) return true;
  return red_mode(p->opts.reduction) == kRedDf && p->opts.cg_variant == 0;
}

// Dynamic shared memory, slot size and grid of a group for its block size and residency: every member's
// layout (K = 0 when streaming), CTAs per SM from the kernel's occupancy (registers, threads, shared memory).
sspcg_status shape_group(const sspcg_plan *p, const GroupSet &set, PcgGroup &g, const std::vector<ProbDesc> &descs) {
  const int cg = set.f64 ? 0 : p->opts.cg_variant;
  const int red = set.f64 ? kRedF64 : red_mode(p->opts.reduction);
  int64_t maxbytes = 0;
  for (int32_t i : g.members) {
    const ProbDesc &d = descs[i];
    int K = 0;
    int64_t b = 0;
    if (g.gvec) {
      b = gvec_slot(set.op, d.N, d.nx, d.nu, p->opts.poly_degree, cg);
    } else {
      const int sched = g.stream ? SSPCG_SCHED_STREAM : p->opts.schedule;
      if (!pcg_fit(set.op, sched, d.N, d.nx, d.nu, set.f64, p->opts.poly_degree, cg, &K, &b, g.stream ? 1 : g.share))
        return SSPCG_ERR_UNSUPPORTED;
    }
    maxbytes = std::max(maxbytes, b);
  }
  int ctas = 0;
  const bool cgv = cg && set.op == kOpQp && !set.f64;
  if (g.warps > 0) {  // one problem per warp: a slot of maxbytes (16-byte multiple) per warp
    const int64_t slot = round_up(maxbytes, 16);
    if (slot * g.warps > smem_budget()) return SSPCG_ERR_UNSUPPORTED;
    g.block = 32 * g.warps;
    cudaError_t e = occupancy_pcg(g.nx, set.op, red, set.f64, false, cgv, true, g.block, (size_t)(slot * g.warps),
                                  &ctas);
    if (e != cudaSuccess) return cuda_fail(e);
    if (ctas < 1) return SSPCG_ERR_UNSUPPORTED;
    g.smem = (size_t)(slot * g.warps);
    g.grid = (int)std::min<int64_t>((g.nwork + g.warps - 1) / g.warps, (int64_t)ctas * device_sms());
    return SSPCG_OK;
  }
  cudaError_t e = occupancy_pcg(g.nx, set.op, red, set.f64, g.gvec, cgv, false, g.block,
                                g.gvec ? 0 : (size_t)maxbytes, &ctas);
  if (e != cudaSuccess) return cuda_fail(e);
  ctas = std::max(1, ctas);
  if (g.gvec) {
    g.smem = 0;
    g.slot_elems = maxbytes;
    g.grid = (int)std::min<int64_t>(g.nwork, (int64_t)std::min(ctas, 2) * device_sms());
    g.grid = std::min(g.grid, g.max_grid);
  } else {
    g.smem = (size_t)maxbytes;
    g.grid = (int)std::min<int64_t>(g.nwork, (int64_t)ctas * device_sms());
  }
  return SSPCG_OK;
}

// PCG launch groups of one set: its members grouped by (nx, residency), each
// group's work list ordered largest first.  ``members`` index ``descs``.
sspcg_status plan_groups(sspcg_plan *p, GroupSet &set, const std::vector<ProbDesc> &descs,
                         const std::vector<int32_t> &members, std::vector<int32_t> &work_host, int32_t &pos) {
  // class 0: not fully resident (takes the whole budget); classes 1..3: fully resident within
  // budget/2, /4, /8 (several CTAs per SM); class 4: the rest of the fully resident problems
  // class 5: vectors in a global workspace (they alone exceed the shared memory)
  constexpr int kClasses = 6;
  std::vector<std::vector<int32_t>> buckets(kClasses * (kMaxNx + 1));
  std::vector<int64_t> bytes(descs.size(), 0);
  const int64_t budget = smem_budget();
  for (int32_t i : members) {
    const ProbDesc &d = descs[i];
    int K = 0;
    if (!pcg_fit(set.op, p->opts.schedule, d.N, d.nx, d.nu, set.f64, p->opts.poly_degree, p->opts.cg_variant, &K,
                 &bytes[i])) {
      if (set.op != kOpQp) {  // global-vector kernels exist for the QP operator form only
        set.unsupported = true;
        continue;
      }
      buckets[kClasses * d.nx + 5].push_back(i);
      continue;
    }
    int cls = 0;
    if (K == d.N + 1) {
      const int64_t need = bytes[i] + kPcgStaticSmem + 1024;
      cls = need * 8 <= budget ? 3 : need * 4 <= budget ? 2 : need * 2 <= budget ? 1 : 4;
    }
    buckets[kClasses * d.nx + cls].push_back(i);
  }
  for (int nx = 1; nx <= kMaxNx; ++nx) {
    for (int r = 0; r < kClasses; ++r) {
      auto &b = buckets[kClasses * nx + r];
      if (b.empty()) continue;
      std::stable_sort(b.begin(), b.end(), [&](int32_t x, int32_t y) { return descs[x].N > descs[y].N; });
      PcgGroup g;
      g.nx = nx;
      g.cls = r;
      g.resident = r != 0 && r != 5;
      g.gvec = r == 5;
      g.f64 = set.f64;
      g.stream = p->opts.schedule == SSPCG_SCHED_STREAM;
      g.members = b;
      for (int32_t i : b) {
        const ProbDesc &d = descs[i];
        g.maxrows = std::max<int64_t>(g.maxrows, (int64_t)(d.N + 1) * d.nx);
        g.maxN = std::max(g.maxN, d.N);
        // bytes per iteration times iterations, which grow about as sqrt(N + 1)
        g.work += std::pow((double)(d.N + 1), 1.5) * d.nx * (3.0 * d.nx + d.nu);
      }
      g.block = p->opts.block_threads > 0 ? p->opts.block_threads : auto_block(g.maxrows);
      g.nwork = (int32_t)b.size();
      if (p->opts.block_threads == 0 && p->opts.schedule == SSPCG_SCHED_AUTO) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(p, set, g));
        if (it != g_tune_cache.end()) {
          g.block = it->second.block;
          g.stream = it->second.stream && r == 0;
          g.share = r == 0 ? it->second.share : 1;
          g.warps = warp_ok(p, set, g) ? it->second.warps : 0;
          g.tuned = true;
        }
      }
      if (p->opts.schedule == SSPCG_SCHED_WARP && warp_ok(p, set, g)) {
        // one problem per warp: as many warps (a power of two, at most 16) as slots of the largest member fit
        int64_t slot = 0;
        for (int32_t i : b) slot = std::max(slot, round_up(bytes[i], 16));
        const int64_t fit = slot > 0 ? smem_budget() / slot : 1;
        g.warps = 1;
        while (g.warps < 16 && 2 * g.warps <= fit) g.warps *= 2;
      }
      if (g.gvec) {
        // two CTAs per SM at most: each holds a workspace slot (about 7 (N+1) nx values)
        g.max_grid = (int)std::min<int64_t>((int64_t)b.size(), 2 * (int64_t)device_sms());
        g.slot_elems = 0;
        for (int32_t i : b)
          g.slot_elems = std::max(g.slot_elems, gvec_slot(set.op, descs[i].N, descs[i].nx, descs[i].nu,
                                                          p->opts.poly_degree, set.f64 ? 0 : p->opts.cg_variant));
        g.scratch_off = set.scratch_elems;
        set.scratch_elems += (int64_t)g.max_grid * g.slot_elems;
      }
      sspcg_status s = shape_group(p, set, g, descs);
      if (s == SSPCG_ERR_UNSUPPORTED && g.warps > 0) {  // a cached warp count whose slots do not fit this group
        g.warps = 0;
        s = shape_group(p, set, g, descs);
      }
      if (s != SSPCG_OK) return s;
      g.d_work = p->d_work + pos;
      g.counter_index = p->ngroups_total++;
      for (int32_t i : b) work_host[pos++] = i;
      (g.gvec ? set.n_gvec : g.resident ? set.n_resident : set.n_stream) += g.nwork;
      set.groups.push_back(std::move(g));
    }
  }
  return SSPCG_OK;
}

PcgArgs make_args(const sspcg_options *o) {
  PcgArgs a{};
  a.tol2 = (float)(o->tol * o->tol);
  a.max_iter = o->max_iter;
  a.warm = o->warm_start;
  a.poly = o->poly_degree;
  a.cg = o->cg_variant;
  a.lambda_f32 = 1;
  a.max_resident = o->schedule == SSPCG_SCHED_STREAM ? 0 : (1 << 30);
  return a;
}

struct SetLaunch {
  const GroupSet *set;
  PcgArgs args;
};

// Vectors of a global-vector group: its part of the plan's workspace (the FP64 set of the pipeline sits
// after the FP32 set's part).
void set_gvec(PcgArgs &a, const sspcg_plan *p, const GroupSet &set, const PcgGroup &g) {
  a.gscratch = nullptr;
  a.gstride = 0;
  if (!g.gvec || !p->d_scratch) return;
  char *base = static_cast<char *>(p->d_scratch);
  if (&set == &p->sets[kSetTiny]) base += p->tiny_scratch_byte_off;
  a.gscratch = base + g.scratch_off * (set.f64 ? sizeof(double) : sizeof(float));
  a.gstride = g.slot_elems;
}

// Launch the groups of several sets concurrently: fork side streams off
// ``st``, one group per stream, join back.
sspcg_status launch_sets(sspcg_plan *p, std::initializer_list<SetLaunch> list, cudaStream_t st) {
  struct Item {
    const PcgGroup *g;
    const PcgArgs *a;
    const GroupSet *set;
  };
  std::vector<Item> all;
  for (const SetLaunch &sl : list)
    for (const PcgGroup &g : sl.set->groups) all.push_back({&g, &sl.args, sl.set});
  if (all.empty()) return SSPCG_OK;
  // heaviest group first: the persistent CTAs of the longest launch take their SMs first and the lighter
  // launches fill in around them, which shortens the tail
  std::stable_sort(all.begin(), all.end(), [](const Item &x, const Item &y) { return x.g->work > y.g->work; });
  SSPCG_CUDA(cudaMemsetAsync(p->d_counters, 0, sizeof(int32_t) * p->ngroups_total, st));
  const size_t ng = all.size();
  if (ng > 1) {
    SSPCG_CUDA(cudaEventRecord(p->ev[0], st));
    for (size_t i = 1; i < ng; ++i) SSPCG_CUDA(cudaStreamWaitEvent(p->side[i - 1], p->ev[0], 0));
  }
  for (size_t i = 0; i < ng; ++i) {
    const PcgGroup &g = *all[i].g;
    PcgArgs a = *all[i].a;
    a.work = g.d_work;
    a.nwork = g.nwork;
    a.counter = p->d_counters + g.counter_index;
    set_gvec(a, p, *all[i].set, g);
    if (g.stream) a.max_resident = 0;
    a.warp = g.warps > 0 ? 1 : 0;
    cudaStream_t s = i == 0 ? st : p->side[i - 1];
    const int red = g.f64 ? kRedF64 : red_mode(p->opts.reduction);
    SSPCG_CUDA(launch_pcg(g.nx, all[i].set->op, red, g.f64, a, g.grid, g.block, g.smem, s));
  }
  for (size_t i = 1; i < ng; ++i) {
    SSPCG_CUDA(cudaEventRecord(p->ev[i], p->side[i - 1]));
    SSPCG_CUDA(cudaStreamWaitEvent(st, p->ev[i], 0));
  }
  return SSPCG_OK;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

// (problem, block row) table of the knots (first = 0) or off-diagonal blocks
// (first = 1) of ``descs``.
std::vector<int2> row_refs(const std::vector<ProbDesc> &descs, int first) {
  std::vector<int2> r;
  for (size_t i = 0; i < descs.size(); ++i)
    for (int k = first; k <= descs[i].N; ++k) r.push_back(make_int2((int)i, k));
  return r;
}

// Split ``members`` of ``descs`` by nx into device descriptor subsets with knot tables.
cudaError_t make_nx_groups(const std::vector<ProbDesc> &descs, const std::vector<int32_t> &members,
                           std::vector<NxGroup> &out) {
  for (int nx = 1; nx <= kMaxNx; ++nx) {
    std::vector<ProbDesc> sub;
    for (int32_t i : members)
      if (descs[i].nx == nx) sub.push_back(descs[i]);
    if (sub.empty()) continue;
    const std::vector<int2> refs = row_refs(sub, 0), orefs = row_refs(sub, 1);
    NxGroup g;
    g.nx = nx;
    for (const ProbDesc &d : sub) g.mx = std::max(g.mx, std::max(d.nx, d.nu));
    g.nprob = (int32_t)sub.size();
    g.knots = (int64_t)refs.size();
    g.offs = (int64_t)orefs.size();
    out.push_back(g);  // pushed first so that plan_free releases partial uploads
    cudaError_t e = upload(&out.back().d_desc, sub);
    if (e == cudaSuccess) e = upload(&out.back().d_refs, refs);
    if (e == cudaSuccess) e = upload(&out.back().d_orefs, orefs);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void time_mark(sspcg_plan *p, int i, cudaStream_t st) {
  if (p->timing) cudaEventRecord(p->tev[i], st);
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
  SSPCG_CUDA(launch_schur_build<float>(ps, nullptr, N + 1, A, B, qd, rd, D, E, (cudaStream_t)stream, device_sms(),
                                       std::max(nx, nu)));
  return SSPCG_OK;
}

sspcg_status sspcg_build_schur_f64(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                                   const float *rd, double *D, double *E, sspcg_stream stream) {
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!qd || !D || (N > 0 && (!A || !rd || !E || (nu > 0 && !B)))) return SSPCG_ERR_INVALID_ARG;
  ProbSet ps{nullptr, single_desc(N, nx, nu), 1};
  SSPCG_CUDA(launch_schur_build<double>(ps, nullptr, N + 1, A, B, qd, rd, D, E, (cudaStream_t)stream, device_sms(),
                                        std::max(nx, nu)));
  return SSPCG_OK;
}

sspcg_status sspcg_build_precond_f64(int32_t N, int32_t nx, sspcg_precond kind, const double *D, const double *E,
                                     double *PD, double *PE, int32_t *status, sspcg_stream stream) {
  if (!shape_ok(N, nx, 0) || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (!D || !PD || !status || (N > 0 && (!E || !PE))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ProbSet ps{nullptr, single_desc(N, nx, 0), 1};
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  SSPCG_CUDA(launch_precond_inv<double>(ps, nullptr, N + 1, nx, (int)kind, D, PD, status, st));
  SSPCG_CUDA(
      launch_precond_off<double>(ps, nullptr, N, (int)kind, E, PD, PE, st, device_sms(), (int64_t)N * nx * nx, nx));
  return SSPCG_OK;
}

sspcg_status sspcg_build_precond(int32_t N, int32_t nx, sspcg_precond kind, const float *D, const float *E,
                                 float *PD, float *PE, int32_t *status, sspcg_stream stream) {
  if (!shape_ok(N, nx, 0) || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (!D || !PD || !status || (N > 0 && (!E || !PE))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ProbSet ps{nullptr, single_desc(N, nx, 0), 1};
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  SSPCG_CUDA(launch_precond_inv<float>(ps, nullptr, N + 1, nx, (int)kind, D, PD, status, st));
  SSPCG_CUDA(
      launch_precond_off<float>(ps, nullptr, N, (int)kind, E, PD, PE, st, device_sms(), (int64_t)N * nx * nx, nx));
  return SSPCG_OK;
}

static sspcg_status solve_single(int op, bool f64, int32_t N, int32_t nx, int32_t nu, const float *A,
                                 const float *B, const float *qd, const float *rd, const float *D, const float *E,
                                 const void *PD, const void *PE, const float *gamma, void *lambda,
                                 const sspcg_options *opts, int32_t *iters, double *relres, int32_t *status,
                                 sspcg_stream stream) {
  if (validate_opts(opts) != SSPCG_OK) return SSPCG_ERR_INVALID_ARG;
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!PD || !gamma || !lambda || !iters || !relres || !status) return SSPCG_ERR_INVALID_ARG;  // PE may be NULL
  if (op == kOpQp && (!qd || (N > 0 && (!A || !rd || (nu > 0 && !B))))) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpBlock && (!D || (N > 0 && !E))) return SSPCG_ERR_INVALID_ARG;
  int K = 0;
  int64_t bytes = 0;
  if (!pcg_fit(op, opts->schedule, N, nx, nu, f64, opts->poly_degree, opts->cg_variant, &K, &bytes))
    return SSPCG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  PcgArgs a = make_args(opts);
  a.ps = ProbSet{nullptr, single_desc(N, nx, nu), 1};
  a.work = nullptr; a.nwork = 1; a.counter = nullptr;
  a.A = A; a.B = B; a.qd = qd; a.rd = rd; a.D = D; a.E = E; a.PD = PD; a.PE = PE;
  a.gamma = gamma; a.lambda = lambda; a.iters = iters; a.relres = relres; a.status = status;
  a.lambda_f32 = f64 ? 0 : 1;
  const int block = opts->block_threads > 0 ? opts->block_threads : auto_block((int64_t)(N + 1) * nx);
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  SSPCG_CUDA(launch_pcg(nx, op, f64 ? kRedF64 : red_mode(opts->reduction), f64, a, 1, block, (size_t)bytes, st));
  return SSPCG_OK;
}

sspcg_status sspcg_solve(int32_t N, int32_t nx, const float *D, const float *E, const float *PD, const float *PE,
                         const float *gamma, float *lambda, const sspcg_options *opts, int32_t *iters,
                         double *relres, int32_t *status, sspcg_stream stream) {
  return solve_single(kOpBlock, false, N, nx, 0, nullptr, nullptr, nullptr, nullptr, D, E, PD, PE, gamma, lambda,
                      opts, iters, relres, status, stream);
}

sspcg_status sspcg_solve_qp(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                            const float *rd, const float *PD, const float *PE, const float *gamma, float *lambda,
                            const sspcg_options *opts, int32_t *iters, double *relres, int32_t *status,
                            sspcg_stream stream) {
  return solve_single(kOpQp, false, N, nx, nu, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, opts, iters,
                      relres, status, stream);
}

sspcg_status sspcg_solve_qp_f64(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                                const float *rd, const double *PD, const double *PE, const float *gamma,
                                double *lambda, const sspcg_options *opts, int32_t *iters, double *relres,
                                int32_t *status, sspcg_stream stream) {
  return solve_single(kOpQp, true, N, nx, nu, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, opts, iters,
                      relres, status, stream);
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
  std::vector<int32_t> all, main_set, tiny;
  for (int32_t i = 0; i < nprob; ++i) {
    const int64_t n = N[i] + 1, m = nx[i], u = nu[i], Ni = N[i];
    const int64_t sz[SSPCG_NUM_ARRAYS] = {Ni * m * m, Ni * m * u, n * m, Ni * u, n * m * m, Ni * m * m, n * m,
                                          Ni * u * u};
    for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) {
      p->offsets[k][i] = cur[k];
      cur[k] += round_up(sz[k], 4);  // 16-byte aligned problem starts
    }
    ProbDesc &d = p->hdesc[i];
    d.N = N[i]; d.nx = nx[i]; d.nu = nu[i]; d.id = i;
    d.oA = p->offsets[SSPCG_ARRAY_A][i];
    d.oB = p->offsets[SSPCG_ARRAY_B][i];
    d.oq = p->offsets[SSPCG_ARRAY_QD][i];
    d.orr = p->offsets[SSPCG_ARRAY_RD][i];
    d.odiag = p->offsets[SSPCG_ARRAY_DIAG][i];
    d.ooff = p->offsets[SSPCG_ARRAY_OFF][i];
    d.ovec = p->offsets[SSPCG_ARRAY_VEC][i];
    knot_start[i + 1] = knot_start[i] + n;
    off_start[i + 1] = off_start[i] + Ni;
    all.push_back(i);
    p->mx = std::max(p->mx, std::max(nx[i], nu[i]));
    const bool f64 = opts->precision == SSPCG_PRECISION_F64 ||
                     (opts->precision == SSPCG_PRECISION_AUTO && n * m <= kTinyUnknowns);
    (f64 ? tiny : main_set).push_back(i);
  }
  for (int k = 0; k < SSPCG_NUM_ARRAYS; ++k) p->sizes[k] = cur[k];
  p->total_knots = knot_start[nprob];
  p->total_off = off_start[nprob];
  p->knot_start = knot_start;
  // FP64 subset: same inputs, FP64 blocks in plan memory
  p->ntiny = (int32_t)tiny.size();
  std::vector<int64_t> tknot(p->ntiny + 1, 0), toff(p->ntiny + 1, 0);
  for (int32_t t = 0; t < p->ntiny; ++t) {
    ProbDesc d = p->hdesc[tiny[t]];
    const int64_t n = d.N + 1, m = d.nx;
    d.odiag = p->t_diag;
    d.ooff = p->t_offe;
    p->t_diag += round_up(n * m * m, 2);
    p->t_offe += round_up((int64_t)d.N * m * m, 2);
    p->tdesc.push_back(d);
    p->mx_tiny = std::max(p->mx_tiny, std::max(d.nx, d.nu));
    tknot[t + 1] = tknot[t] + n;
    toff[t + 1] = toff[t] + d.N;
  }
  p->tknots = tknot[p->ntiny];
  p->toff = toff[p->ntiny];
  auto fail = [&](sspcg_status s) { plan_free(p); return s; };
  if (nprob > 0) {
    cudaError_t e;
    if ((e = upload(&p->d_desc, p->hdesc)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = upload(&p->d_kref, row_refs(p->hdesc, 0))) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = upload(&p->d_oref, row_refs(p->hdesc, 1))) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = upload(&p->d_knot_start, p->knot_start)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = make_nx_groups(p->hdesc, all, p->nxg_all)) != cudaSuccess) return fail(cuda_fail(e));
    if (p->ntiny > 0) {
      std::vector<int32_t> tl(p->ntiny);
      std::iota(tl.begin(), tl.end(), 0);
      if ((e = make_nx_groups(p->tdesc, tl, p->nxg_tiny)) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = upload(&p->d_tdesc, p->tdesc)) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = upload(&p->d_tkref, row_refs(p->tdesc, 0))) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = upload(&p->d_toref, row_refs(p->tdesc, 1))) != cudaSuccess) return fail(cuda_fail(e));
      const int64_t td = std::max<int64_t>(p->t_diag, 2), to = std::max<int64_t>(p->t_offe, 2);
      if ((e = cudaMalloc(&p->D64, sizeof(double) * td)) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = cudaMalloc(&p->PD64, sizeof(double) * td)) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = cudaMalloc(&p->E64, sizeof(double) * to)) != cudaSuccess) return fail(cuda_fail(e));
      if ((e = cudaMalloc(&p->PE64, sizeof(double) * to)) != cudaSuccess) return fail(cuda_fail(e));
    }
    const size_t nwork = 2 * (size_t)nprob + main_set.size() + tiny.size();
    if ((e = cudaMalloc(&p->d_work, sizeof(int32_t) * nwork)) != cudaSuccess) return fail(cuda_fail(e));
    std::vector<int32_t> work(nwork);
    std::vector<int32_t> tiny_local(p->ntiny);
    std::iota(tiny_local.begin(), tiny_local.end(), 0);
    int32_t pos = 0;
    for (int k = 0; k < kNumSets; ++k) p->sets[k].id = k;
    p->sets[kSetQpAll].op = kOpQp;
    p->sets[kSetBlockAll].op = kOpBlock;
    p->sets[kSetQpMain].op = kOpQp;
    p->sets[kSetTiny].op = kOpQp;
    p->sets[kSetTiny].f64 = true;
    sspcg_status s;
    if ((s = plan_groups(p, p->sets[kSetQpAll], p->hdesc, all, work, pos)) != SSPCG_OK) return fail(s);
    if ((s = plan_groups(p, p->sets[kSetBlockAll], p->hdesc, all, work, pos)) != SSPCG_OK) return fail(s);
    if ((s = plan_groups(p, p->sets[kSetQpMain], p->hdesc, main_set, work, pos)) != SSPCG_OK) return fail(s);
    if ((s = plan_groups(p, p->sets[kSetTiny], p->tdesc, tiny_local, work, pos)) != SSPCG_OK) return fail(s);
    if ((e = cudaMemcpy(p->d_work, work.data(), sizeof(int32_t) * nwork, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e));
    {
      // padded copies for the problems of the QP-form set that do not fit in shared memory whole (and, under
      // the STREAM schedule, for every problem): N nx (2 vec_stride(nx) + vec_stride(nu)) floats each
      std::vector<int64_t> off(nprob, -1);
      std::vector<int32_t> list;
      int64_t total = 0;
      for (const PcgGroup &g : p->sets[kSetQpAll].groups) {
        if (!(g.cls == 0 || g.cls == 5 || p->opts.schedule == SSPCG_SCHED_STREAM)) continue;
        for (int32_t i : g.members) {
          const ProbDesc &d = p->hdesc[i];
          if (d.N == 0) continue;
          off[d.id] = total;
          list.push_back(i);
          const int64_t rows = (int64_t)d.N * d.nx;
          total += 2 * pad_region(rows, d.nx) + pad_region(rows, d.nu);  // multiples of 8 floats
        }
      }
      p->npad = (int32_t)list.size();
      if (p->npad > 0) {
        if ((e = cudaMalloc(&p->d_pad, sizeof(float) * total)) != cudaSuccess) return fail(cuda_fail(e));
        if ((e = upload(&p->d_pad_off, off)) != cudaSuccess) return fail(cuda_fail(e));
        if ((e = upload(&p->d_pad_list, list)) != cudaSuccess) return fail(cuda_fail(e));
      }
    }
    {
      // bytes: the largest set alone, or the pipeline's FP32 and FP64 sets side by side
      const int64_t b32 = (int64_t)sizeof(float), b64 = (int64_t)sizeof(double);
      auto sb = [&](int k) { return p->sets[k].scratch_elems * (p->sets[k].f64 ? b64 : b32); };
      const int64_t main_bytes = round_up(sb(kSetQpMain), 64);
      int64_t need = std::max({sb(kSetQpAll), sb(kSetBlockAll), main_bytes + sb(kSetTiny)});
      p->tiny_scratch_byte_off = main_bytes;
      if (need > 0 && (e = cudaMalloc(&p->d_scratch, need)) != cudaSuccess) return fail(cuda_fail(e));
    }
    if ((e = cudaMalloc(&p->d_counters, sizeof(int32_t) * std::max(1, p->ngroups_total))) != cudaSuccess)
      return fail(cuda_fail(e));
    size_t nside = 0;
    for (int k = 0; k < kNumSets; ++k) nside = std::max(nside, p->sets[k].groups.size());
    nside = std::max(nside, p->sets[kSetQpMain].groups.size() + p->sets[kSetTiny].groups.size());
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
  const GroupSet &m = plan->sets[kSetQpMain], &t = plan->sets[kSetTiny];
  out[0] = (int64_t)(m.groups.size() + t.groups.size());
  out[1] = m.n_resident;
  out[2] = m.n_stream + m.n_gvec;
  out[3] = plan->ntiny;
  out[4] = (int64_t)plan->sets[kSetQpAll].groups.size();
  out[5] = (int64_t)plan->sets[kSetBlockAll].groups.size();
  out[6] = plan->sets[kSetQpAll].n_resident;
  out[7] = plan->sets[kSetQpAll].n_stream + plan->sets[kSetQpAll].n_gvec;
  return SSPCG_OK;
}

sspcg_status sspcg_plan_set_timing(sspcg_plan *plan, int32_t enable) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (enable && !plan->tev[0])
    for (auto &e : plan->tev) SSPCG_CUDA(cudaEventCreate(&e));
  plan->timing = enable != 0;
  return SSPCG_OK;
}

sspcg_status sspcg_plan_timings(sspcg_plan *plan, float *out_ms) {
  if (!plan || !out_ms || !plan->tev[0]) return SSPCG_ERR_INVALID_ARG;
  SSPCG_CUDA(cudaEventSynchronize(plan->tev[2]));
  out_ms[0] = 0.0f;
  if (plan->build_timed) SSPCG_CUDA(cudaEventElapsedTime(&out_ms[0], plan->tev[0], plan->tev[1]));
  SSPCG_CUDA(cudaEventElapsedTime(&out_ms[1], plan->tev[1], plan->tev[2]));
  return SSPCG_OK;
}

static ProbSet plan_set(const sspcg_plan *p) { return ProbSet{p->d_desc, ProbDesc{}, p->nprob}; }
static ProbSet tiny_set(const sspcg_plan *p) { return ProbSet{p->d_tdesc, ProbDesc{}, p->ntiny}; }

sspcg_status sspcg_build_schur_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                       const float *rd, float *D, float *E, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!qd || !D || !aligned16(qd) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  if (plan->total_off > 0 && (!A || !rd || !E || !B)) return SSPCG_ERR_INVALID_ARG;
  SSPCG_CUDA(launch_schur_build<float>(plan_set(plan), plan->d_kref, plan->total_knots, A, B, qd, rd, D, E,
                                       (cudaStream_t)stream, device_sms(), plan->mx));
  return SSPCG_OK;
}

static int64_t schur_full_work(int32_t N, int32_t nx, int32_t nu) {
  return round_up((int64_t)(N + 1) * nx * nx, 4) + (int64_t)N * nu * nu;
}

sspcg_status sspcg_schur_full_work_floats(int32_t N, int32_t nx, int32_t nu, int64_t *floats) {
  if (!floats || !shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  *floats = schur_full_work(N, nx, nu);
  return SSPCG_OK;
}

sspcg_status sspcg_build_schur_full(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *Q,
                                    const float *R, float *D, float *E, float *work, int32_t *status,
                                    sspcg_stream stream) {
  if (!shape_ok(N, nx, nu)) return SSPCG_ERR_INVALID_ARG;
  if (!Q || !D || !work || !status || (N > 0 && (!A || !E || (nu > 0 && (!B || !R))))) return SSPCG_ERR_INVALID_ARG;
  if (!aligned16(work)) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *qi = work, *ri = work + round_up((int64_t)(N + 1) * nx * nx, 4);
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  // Q_k^-1 and R_k^-1 by the FP64 LDL^T inversion of the preconditioner build (Q is laid out like D; the R
  // blocks are N blocks of nu x nu, that is, the diagonal blocks of a problem with nx = nu and N - 1)
  SSPCG_CUDA(launch_precond_inv<float>(ProbSet{nullptr, single_desc(N, nx, nu), 1}, nullptr, N + 1, nx,
                                       (int)SSPCG_PRECOND_SYM_STAIR, Q, qi, status, st));
  if (N > 0 && nu > 0)
    SSPCG_CUDA(launch_precond_inv<float>(ProbSet{nullptr, single_desc(N - 1, nu, 0), 1}, nullptr, N, nu,
                                         (int)SSPCG_PRECOND_SYM_STAIR, R, ri, status, st));
  SSPCG_CUDA(launch_schur_full(ProbSet{nullptr, single_desc(N, nx, nu), 1}, nullptr, N + 1, nullptr, A, B, qi, ri, D,
                               E, st, std::max(nx, nu)));
  return SSPCG_OK;
}

static sspcg_status full_setup(sspcg_plan *p) {
  if (p->full_ready) return SSPCG_OK;
  SSPCG_CUDA(cudaMalloc(&p->qinv, sizeof(float) * std::max<int64_t>(p->sizes[SSPCG_ARRAY_DIAG], 4)));
  SSPCG_CUDA(cudaMalloc(&p->rinv, sizeof(float) * std::max<int64_t>(p->sizes[SSPCG_ARRAY_RFULL], 4)));
  SSPCG_CUDA(upload(&p->d_roff, p->offsets[SSPCG_ARRAY_RFULL]));
  // the R blocks of problem i as the diagonal blocks of a problem with nx = nu and N - 1 block rows
  std::vector<ProbDesc> rd(p->hdesc);
  std::vector<int32_t> members;
  for (int32_t i = 0; i < p->nprob; ++i) {
    ProbDesc &d = rd[i];
    if (d.N > 0 && d.nu > 0) members.push_back(i);
    d.odiag = p->offsets[SSPCG_ARRAY_RFULL][i];
    d.nx = d.nu > 0 ? d.nu : 1;
    d.N = d.N - 1;
    d.nu = 0;
  }
  SSPCG_CUDA(make_nx_groups(rd, members, p->nxg_r));
  p->full_ready = true;
  return SSPCG_OK;
}

sspcg_status sspcg_build_schur_full_batched(sspcg_plan *plan, const float *A, const float *B, const float *Q,
                                            const float *R, float *D, float *E, int32_t *status,
                                            sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!Q || !D || !status || !aligned16(Q) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  if (plan->total_off > 0 && (!A || !B || !E)) return SSPCG_ERR_INVALID_ARG;
  if (plan->sizes[SSPCG_ARRAY_RFULL] > 0 && !R) return SSPCG_ERR_INVALID_ARG;
  sspcg_status s = full_setup(plan);
  if (s != SSPCG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  for (const NxGroup &g : plan->nxg_all)
    SSPCG_CUDA(launch_precond_inv<float>(ProbSet{g.d_desc, ProbDesc{}, g.nprob}, g.d_refs, g.knots, g.nx,
                                         (int)SSPCG_PRECOND_SYM_STAIR, Q, plan->qinv, status, st));
  for (const NxGroup &g : plan->nxg_r)
    SSPCG_CUDA(launch_precond_inv<float>(ProbSet{g.d_desc, ProbDesc{}, g.nprob}, g.d_refs, g.knots, g.nx,
                                         (int)SSPCG_PRECOND_SYM_STAIR, R, plan->rinv, status, st));
  SSPCG_CUDA(launch_schur_full(plan_set(plan), plan->d_kref, plan->total_knots, plan->d_roff, A, B, plan->qinv,
                               plan->rinv, D, E, st, plan->mx));
  return SSPCG_OK;
}

sspcg_status sspcg_build_precond_batched(sspcg_plan *plan, sspcg_precond kind, const float *D, const float *E,
                                         float *PD, float *PE, int32_t *status, sspcg_stream stream) {
  if (!plan || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!D || !PD || !status || (plan->total_off > 0 && (!E || !PE))) return SSPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  for (const NxGroup &g : plan->nxg_all)
    SSPCG_CUDA(launch_precond_inv<float>(ProbSet{g.d_desc, ProbDesc{}, g.nprob}, g.d_refs, g.knots, g.nx,
                                         (int)kind, D, PD, status, st));
  SSPCG_CUDA(launch_precond_off<float>(plan_set(plan), plan->d_oref, plan->total_off, (int)kind, E, PD, PE, st,
                                       device_sms(), plan->sizes[SSPCG_ARRAY_OFF], plan->mx));
  return SSPCG_OK;
}

static PcgArgs batched_args(sspcg_plan *plan, const float *A, const float *B, const float *qd, const float *rd,
                            const float *D, const float *E, const void *PD, const void *PE, const float *gamma,
                            float *lambda, int32_t *iters, double *relres, int32_t *status) {
  PcgArgs a = make_args(&plan->opts);
  a.ps = plan_set(plan);
  a.A = A; a.B = B; a.qd = qd; a.rd = rd; a.D = D; a.E = E; a.PD = PD; a.PE = PE;
  a.gamma = gamma; a.lambda = lambda; a.iters = iters; a.relres = relres; a.status = status;
  return a;
}

// Padded copies of the streamed problems' A, B and PE (PE nullptr: block-diagonal preconditioner, no copy), on
// st before the PCG launches of a QP-form FP32 set, and the launch arguments that point the kernel at them.
static sspcg_status pad_streamed(sspcg_plan *plan, const float *A, const float *B, const float *PE, PcgArgs &a,
                                 cudaStream_t st) {
  if (plan->npad == 0) return SSPCG_OK;
  SSPCG_CUDA(launch_pad_rows(plan->d_desc, plan->d_pad_list, plan->npad, A, B, PE, plan->d_pad_off, plan->d_pad,
                             device_sms(), st));
  a.pad = plan->d_pad;
  a.pad_off = plan->d_pad_off;
  return SSPCG_OK;
}

static sspcg_status check_solve_args(sspcg_plan *plan, int op, const float *A, const float *B, const float *qd,
                                     const float *rd, const float *D, const float *E, const float *PD,
                                     const float *PE, const float *gamma, float *lambda, int32_t *iters,
                                     double *relres, int32_t *status) {
  if (!PD || !gamma || !lambda || !iters || !relres || !status) return SSPCG_ERR_INVALID_ARG;  // PE may be NULL
  if (op == kOpQp && (!qd || (plan->total_off > 0 && (!A || !rd || !B)))) return SSPCG_ERR_INVALID_ARG;
  if (op == kOpBlock && (!D || (plan->total_off > 0 && !E))) return SSPCG_ERR_INVALID_ARG;
  return SSPCG_OK;
}

sspcg_status sspcg_solve_batched(sspcg_plan *plan, const float *D, const float *E, const float *PD,
                                 const float *PE, const float *gamma, float *lambda, int32_t *iters,
                                 double *relres, int32_t *status, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  sspcg_status s = check_solve_args(plan, kOpBlock, nullptr, nullptr, nullptr, nullptr, D, E, PD, PE, gamma, lambda,
                                    iters, relres, status);
  if (s != SSPCG_OK) return s;
  if (plan->sets[kSetBlockAll].unsupported) return SSPCG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  plan->build_timed = false;
  time_mark(plan, 1, st);
  s = launch_sets(plan, {{&plan->sets[kSetBlockAll], batched_args(plan, nullptr, nullptr, nullptr, nullptr, D, E, PD,
                                                                   PE, gamma, lambda, iters, relres, status)}},
                  st);
  time_mark(plan, 2, st);
  return s;
}

sspcg_status sspcg_solve_qp_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                    const float *rd, const float *PD, const float *PE, const float *gamma,
                                    float *lambda, int32_t *iters, double *relres, int32_t *status,
                                    sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  sspcg_status s = check_solve_args(plan, kOpQp, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters,
                                    relres, status);
  if (s != SSPCG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SSPCG_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * plan->nprob, st));
  plan->build_timed = false;
  time_mark(plan, 1, st);
  PcgArgs a = batched_args(plan, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters, relres, status);
  if ((s = pad_streamed(plan, A, B, PE, a, st)) != SSPCG_OK) return s;
  s = launch_sets(plan, {{&plan->sets[kSetQpAll], a}}, st);
  time_mark(plan, 2, st);
  return s;
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

// First half of the pipeline: FP32 blocks for every problem (also returned to the caller), FP64 blocks for
// the FP64 subset.
static sspcg_status pipeline_build(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                   const float *qd, const float *rd, float *D, float *E, float *PD, float *PE,
                                   int32_t *status, sspcg_stream stream) {
  sspcg_status s;
  cudaStream_t st = (cudaStream_t)stream;
  time_mark(plan, 0, st);
  if ((s = sspcg_build_schur_batched(plan, A, B, qd, rd, D, E, stream)) != SSPCG_OK) return s;
  if ((s = sspcg_build_precond_batched(plan, kind, D, E, PD, PE, status, stream)) != SSPCG_OK) return s;
  if (plan->ntiny > 0) {
    SSPCG_CUDA(launch_schur_build<double>(tiny_set(plan), plan->d_tkref, plan->tknots, A, B, qd, rd, plan->D64,
                                          plan->E64, st, device_sms(), plan->mx_tiny));
    for (const NxGroup &g : plan->nxg_tiny)
      SSPCG_CUDA(launch_precond_inv<double>(ProbSet{g.d_desc, ProbDesc{}, g.nprob}, g.d_refs, g.knots, g.nx,
                                            (int)kind, plan->D64, plan->PD64, status, st));
    SSPCG_CUDA(launch_precond_off<double>(tiny_set(plan), plan->d_toref, plan->toff, (int)kind, plan->E64,
                                          plan->PD64, plan->PE64, st, device_sms(), plan->t_offe, plan->mx_tiny));
  }
  plan->build_timed = true;
  return SSPCG_OK;
}

// Second half: the PCG launches of the FP32 set and the FP64 subset (``warm`` overrides the plan's
// warm-start option).
static sspcg_status pipeline_solve(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                   const float *rd, const float *gamma, const float *PD, const float *PE,
                                   float *lambda, int32_t *iters, double *relres, int32_t *status, int warm,
                                   sspcg_stream stream, bool diag_only = false) {
  cudaStream_t st = (cudaStream_t)stream;
  time_mark(plan, 1, st);
  // block-Jacobi and Jacobi: the off-diagonal blocks are zero, so the solves neither stage nor read them
  PcgArgs a32 = batched_args(plan, A, B, qd, rd, nullptr, nullptr, PD, diag_only ? nullptr : PE, gamma, lambda, iters,
                             relres, status);
  a32.warm = warm;
  PcgArgs a64 = a32;
  a64.ps = tiny_set(plan);
  a64.PD = plan->PD64;
  a64.PE = diag_only ? nullptr : plan->PE64;
  sspcg_status s = pad_streamed(plan, A, B, diag_only ? nullptr : PE, a32, st);
  if (s != SSPCG_OK) return s;
  s = launch_sets(plan, {{&plan->sets[kSetQpMain], a32}, {&plan->sets[kSetTiny], a64}}, st);
  time_mark(plan, 2, st);
  return s;
}

sspcg_status sspcg_pipeline_batched(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                    const float *qd, const float *rd, const float *gamma, float *D, float *E,
                                    float *PD, float *PE, float *lambda, int32_t *iters, double *relres,
                                    int32_t *status, sspcg_stream stream) {
  if (!plan || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  sspcg_status s = check_solve_args(plan, kOpQp, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters,
                                    relres, status);
  if (s != SSPCG_OK) return s;
  if (!D || (plan->total_off > 0 && !E)) return SSPCG_ERR_INVALID_ARG;
  if (!aligned16(qd) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  s = pipeline_build(plan, kind, A, B, qd, rd, D, E, PD, PE, status, stream);
  if (s != SSPCG_OK) return s;
  return pipeline_solve(plan, A, B, qd, rd, gamma, PD, PE, lambda, iters, relres, status, plan->opts.warm_start,
                        stream, kind == SSPCG_PRECOND_BLOCK_JACOBI || kind == SSPCG_PRECOND_JACOBI);
}

sspcg_status sspcg_plan_capture_pipeline(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                         const float *qd, const float *rd, const float *gamma, float *D, float *E,
                                         float *PD, float *PE, float *lambda, int32_t *iters, double *relres,
                                         int32_t *status, sspcg_stream stream) {
  if (!plan || !stream) return SSPCG_ERR_INVALID_ARG;  // capture needs a non-default stream
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->graph) {
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  const bool timing = plan->timing;
  plan->timing = false;
  // run once uncaptured so that every kernel attribute is set before capture
  sspcg_status s = sspcg_pipeline_batched(plan, kind, A, B, qd, rd, gamma, D, E, PD, PE, lambda, iters, relres,
                                          status, stream);
  if (s != SSPCG_OK) { plan->timing = timing; return s; }
  SSPCG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  s = sspcg_pipeline_batched(plan, kind, A, B, qd, rd, gamma, D, E, PD, PE, lambda, iters, relres, status, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  plan->timing = timing;
  if (s != SSPCG_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(&plan->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { plan->graph = nullptr; return cuda_fail(e); }
  return SSPCG_OK;
}

sspcg_status sspcg_plan_launch(sspcg_plan *plan, sspcg_stream stream) {
  if (!plan || !plan->graph) return SSPCG_ERR_INVALID_ARG;
  SSPCG_CUDA(cudaGraphLaunch(plan->graph, (cudaStream_t)stream));
  return SSPCG_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
namespace {

// Time one group alone on ``st``: statuses restored and the work counter cleared before each launch; the
// first launch warms, the best of the next two counts.
sspcg_status time_group(sspcg_plan *p, const GroupSet &set, const PcgGroup &g, const PcgArgs &base,
                        const int32_t *status0, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  PcgArgs a = base;
  a.work = g.d_work;
  a.nwork = g.nwork;
  a.counter = p->d_counters + g.counter_index;
  set_gvec(a, p, set, g);
  if (g.stream) a.max_resident = 0;
  a.warp = g.warps > 0 ? 1 : 0;
  const int red = g.f64 ? kRedF64 : red_mode(p->opts.reduction);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    SSPCG_CUDA(cudaMemcpyAsync(a.status, status0, sizeof(int32_t) * p->nprob, cudaMemcpyDeviceToDevice, st));
    SSPCG_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int32_t), st));
    SSPCG_CUDA(cudaEventRecord(e0, st));
    SSPCG_CUDA(launch_pcg(g.nx, set.op, red, g.f64, a, g.grid, g.block, g.smem, st));
    SSPCG_CUDA(cudaEventRecord(e1, st));
    SSPCG_CUDA(cudaEventSynchronize(e1));
    float t = 0.0f;
    SSPCG_CUDA(cudaEventElapsedTime(&t, e0, e1));
    if (rep > 0) best = std::min(best, t);
  }
  *ms = best;
  return SSPCG_OK;
}

// Every candidate (block size; for partially staged groups also streaming every block row) of every group of
// one set, timed alone; the fastest is kept in the plan and in the process-wide cache.
sspcg_status tune_set(sspcg_plan *p, GroupSet &set, const std::vector<ProbDesc> &descs, const PcgArgs &base,
                      const int32_t *status0, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  static const int kBlocks[] = {64, 96, 128, 160, 192, 256, 320, 384, 448, 512};
  for (PcgGroup &g : set.groups) {
    const PcgGroup orig = g;
    float best_ms = 0.0f;
    sspcg_status s = time_group(p, set, g, base, status0, st, e0, e1, &best_ms);
    if (s != SSPCG_OK) return s;
    PcgGroup best = g;
    // from at most 16 rows per thread to at most one
    const int64_t max_block = std::max<int64_t>(64, round_up(g.maxrows, 32));
    const int64_t min_block = std::min<int64_t>(max_block, g.maxrows / 16);
    // residency candidates: partially staged groups may stage into 1/2 .. 1/4 of the shared memory (several
    // CTAs per SM) or stream every block row; the other classes keep their staging
    for (int cand = 0; cand < (g.cls == 0 ? 5 : 1); ++cand) {
      const bool stream = cand == 4;
      const int share = cand < 4 ? cand + 1 : 1;
      for (int blk : kBlocks) {
        if (blk > max_block || blk < min_block ||
            (blk == orig.block && stream == orig.stream && share == orig.share))
          continue;
        PcgGroup c = orig;
        c.block = blk;
        c.stream = stream;
        c.share = share;
        s = shape_group(p, set, c, descs);
        if (s == SSPCG_ERR_UNSUPPORTED) continue;  // the vectors do not fit in that share
        if (s != SSPCG_OK) return s;
        float ms = 0.0f;
        if ((s = time_group(p, set, c, base, status0, st, e0, e1, &ms)) != SSPCG_OK) return s;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    // fully staged groups: one problem per warp, 1 .. 16 warps per CTA (as many as fit in the budget)
    if (warp_ok(p, set, orig)) {
      for (int w : {1, 2, 4, 8, 16}) {
        PcgGroup c = orig;
        c.warps = w;
        c.stream = false;
        c.share = 1;
        s = shape_group(p, set, c, descs);
        if (s == SSPCG_ERR_UNSUPPORTED) break;  // w slots do not fit
        if (s != SSPCG_OK) return s;
        float ms = 0.0f;
        if ((s = time_group(p, set, c, base, status0, st, e0, e1, &ms)) != SSPCG_OK) return s;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    g = best;
    g.tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(p, set, g)] = TuneChoice{g.block, g.stream, g.share, g.warps};
  }
  return SSPCG_OK;
}

}  // namespace

sspcg_status sspcg_plan_autotune(sspcg_plan *plan, int32_t which, sspcg_precond kind, const float *A, const float *B,
                                 const float *qd, const float *rd, const float *gamma, float *D, float *E, float *PD,
                                 float *PE, float *lambda, int32_t *iters, double *relres, int32_t *status,
                                 sspcg_stream stream) {
  if (!plan || kind < 0 || kind > 3 || which < 1 || which > 3) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  sspcg_status s = check_solve_args(plan, kOpQp, A, B, qd, rd, nullptr, nullptr, PD, PE, gamma, lambda, iters,
                                    relres, status);
  if (s != SSPCG_OK) return s;
  if (!D || (plan->total_off > 0 && !E)) return SSPCG_ERR_INVALID_ARG;
  if (!aligned16(qd) || !aligned16(D)) return SSPCG_ERR_INVALID_ARG;
  // the launch parameters change: a captured pipeline has to be captured again
  if (plan->graph) {
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool timing = plan->timing;
  plan->timing = false;
  s = pipeline_build(plan, kind, A, B, qd, rd, D, E, PD, PE, status, stream);
  plan->timing = timing;
  if (s != SSPCG_OK) return s;
  int32_t *status0 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&status0, sizeof(int32_t) * plan->nprob);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status0, status, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    // block-Jacobi and Jacobi: time the solves without off-diagonal blocks, as the pipeline runs them
    const bool diag_only = kind == SSPCG_PRECOND_BLOCK_JACOBI || kind == SSPCG_PRECOND_JACOBI;
    PcgArgs a32 = batched_args(plan, A, B, qd, rd, nullptr, nullptr, PD, diag_only ? nullptr : PE, gamma, lambda,
                               iters, relres, status);
    a32.warm = 0;
    PcgArgs a64 = a32;
    a64.ps = tiny_set(plan);
    a64.PD = plan->PD64;
    a64.PE = diag_only ? nullptr : plan->PE64;
    s = pad_streamed(plan, A, B, diag_only ? nullptr : PE, a32, st);

    if (s == SSPCG_OK && (which & SSPCG_TUNE_PIPELINE)) {
      s = tune_set(plan, plan->sets[kSetQpMain], plan->hdesc, a32, status0, st, e0, e1);
      if (s == SSPCG_OK) s = tune_set(plan, plan->sets[kSetTiny], plan->tdesc, a64, status0, st, e0, e1);
    }
    if (s == SSPCG_OK && (which & SSPCG_TUNE_SOLVE))
      s = tune_set(plan, plan->sets[kSetQpAll], plan->hdesc, a32, status0, st, e0, e1);
    if (s == SSPCG_OK) e = cudaMemcpyAsync(status, status0, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToDevice, st);
    if (s == SSPCG_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(status0);
  if (s != SSPCG_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e);
  return SSPCG_OK;
}

sspcg_status sspcg_plan_schedule(const sspcg_plan *plan, int32_t which, int32_t *out, int32_t capacity,
                                 int32_t *count) {
  if (!plan || !count || which < 0 || which > 2 || capacity < 0 || (capacity > 0 && !out))
    return SSPCG_ERR_INVALID_ARG;
  const GroupSet &set = plan->sets[which == 0 ? kSetQpMain : which == 1 ? kSetTiny : kSetQpAll];
  *count = (int32_t)set.groups.size();
  const int32_t n = std::min<int32_t>(capacity, *count);
  for (int32_t i = 0; i < n; ++i) {
    const PcgGroup &g = set.groups[i];
    int32_t *r = out + (int64_t)i * SSPCG_SCHEDULE_FIELDS;
    r[0] = g.nx; r[1] = g.cls; r[2] = g.nwork; r[3] = g.maxN; r[4] = g.block; r[5] = g.grid;
    r[6] = (int32_t)g.smem; r[7] = g.stream ? 1 : 0; r[8] = g.tuned ? 1 : 0; r[9] = g.share; r[10] = g.warps;
  }
  return SSPCG_OK;
}

sspcg_status sspcg_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
  return SSPCG_OK;
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

// Asynchronous host pipeline: call i copies its inputs into slot i % 2 on the plan's copy stream (after
// the compute that last read that slot), computes on ``stream`` (after its copies and after the copy-out
// that last read that slot's outputs), and copies its results out on the plan's second copy stream.  So
// the copies of one call overlap the compute of the previous one.
static sspcg_status async_setup(sspcg_plan *p) {
  const int64_t *sz = p->sizes;
  auto r4 = [](int64_t n) { return round_up(std::max<int64_t>(n, 4), 4); };
  if (!p->ablocks) {
    SSPCG_CUDA(cudaMalloc(&p->ablocks, sizeof(float) * (2 * r4(sz[SSPCG_ARRAY_DIAG]) + 2 * r4(sz[SSPCG_ARRAY_OFF]))));
    SSPCG_CUDA(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking));
    SSPCG_CUDA(cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking));
    const int64_t in = r4(sz[SSPCG_ARRAY_A]) + r4(sz[SSPCG_ARRAY_B]) + r4(sz[SSPCG_ARRAY_QD]) + r4(sz[SSPCG_ARRAY_RD]) +
                       2 * r4(sz[SSPCG_ARRAY_VEC]);
    for (auto &a : p->aslot) {
      SSPCG_CUDA(cudaMalloc(&a.buf, sizeof(float) * in));
      SSPCG_CUDA(cudaMalloc(&a.ints, sizeof(int32_t) * 2 * p->nprob));
      SSPCG_CUDA(cudaMalloc(&a.dbl, sizeof(double) * p->nprob));
      for (cudaEvent_t *e : {&a.in_ready, &a.consumed, &a.computed, &a.out_done})
        SSPCG_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
  }
  return SSPCG_OK;
}

sspcg_status sspcg_pipeline_host_async(sspcg_plan *plan, sspcg_precond kind, const float *A_host,
                                       const float *B_host, const float *qd_host, const float *rd_host,
                                       const float *gamma_host, float *lambda_host, int32_t *iters_host,
                                       double *relres_host, int32_t *status_host, sspcg_stream stream) {
  if (!plan || kind < 0 || kind > 3) return SSPCG_ERR_INVALID_ARG;
  if (plan->nprob == 0) return SSPCG_OK;
  if (!qd_host || !gamma_host || !lambda_host || !iters_host || !relres_host || !status_host)
    return SSPCG_ERR_INVALID_ARG;
  sspcg_status s = async_setup(plan);
  if (s != SSPCG_OK) return s;
  const int64_t *sz = plan->sizes;
  auto r4 = [](int64_t n) { return round_up(std::max<int64_t>(n, 4), 4); };
  sspcg_plan::AsyncSlot &a = plan->aslot[plan->acalls & 1];
  float *cur = a.buf;
  auto take = [&](int64_t n) { float *r = cur; cur += r4(n); return r; };
  float *A = take(sz[SSPCG_ARRAY_A]), *B = take(sz[SSPCG_ARRAY_B]), *qd = take(sz[SSPCG_ARRAY_QD]);
  float *rd = take(sz[SSPCG_ARRAY_RD]), *g = take(sz[SSPCG_ARRAY_VEC]), *lam = take(sz[SSPCG_ARRAY_VEC]);
  float *D = plan->ablocks, *E = D + r4(sz[SSPCG_ARRAY_DIAG]), *PD = E + r4(sz[SSPCG_ARRAY_OFF]);
  float *PE = PD + r4(sz[SSPCG_ARRAY_DIAG]);
  int32_t *iters = a.ints, *status = a.ints + plan->nprob;
  double *relres = a.dbl;
  cudaStream_t st = (cudaStream_t)stream;
  // inputs: after the compute that last read this slot
  SSPCG_CUDA(cudaStreamWaitEvent(plan->h2d, a.consumed, 0));
  auto h2d = [&](float *dst, const float *src, int64_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice, plan->h2d);
  };
  cudaError_t e;
  if ((e = h2d(A, A_host, sz[SSPCG_ARRAY_A])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(B, B_host, sz[SSPCG_ARRAY_B])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(qd, qd_host, sz[SSPCG_ARRAY_QD])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(rd, rd_host, sz[SSPCG_ARRAY_RD])) != cudaSuccess) return cuda_fail(e);
  if ((e = h2d(g, gamma_host, sz[SSPCG_ARRAY_VEC])) != cudaSuccess) return cuda_fail(e);
  if (plan->opts.warm_start && (e = h2d(lam, lambda_host, sz[SSPCG_ARRAY_VEC])) != cudaSuccess) return cuda_fail(e);
  SSPCG_CUDA(cudaEventRecord(a.in_ready, plan->h2d));
  // compute: after its inputs, after the copy-out that last read this slot's outputs, and after the
  // previous call's compute (the D, E, PD, PE blocks are shared), whatever stream that one ran on
  SSPCG_CUDA(cudaStreamWaitEvent(st, a.in_ready, 0));
  SSPCG_CUDA(cudaStreamWaitEvent(st, a.out_done, 0));
  SSPCG_CUDA(cudaStreamWaitEvent(st, plan->aslot[(plan->acalls + 1) & 1].computed, 0));
  s = sspcg_pipeline_batched(plan, kind, A, B, qd, rd, g, D, E, PD, PE, lam, iters, relres, status, stream);
  if (s != SSPCG_OK) return s;
  SSPCG_CUDA(cudaEventRecord(a.consumed, st));
  SSPCG_CUDA(cudaEventRecord(a.computed, st));
  // outputs
  SSPCG_CUDA(cudaStreamWaitEvent(plan->d2h, a.computed, 0));
  SSPCG_CUDA(cudaMemcpyAsync(lambda_host, lam, sizeof(float) * sz[SSPCG_ARRAY_VEC], cudaMemcpyDeviceToHost,
                             plan->d2h));
  SSPCG_CUDA(cudaMemcpyAsync(iters_host, iters, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToHost, plan->d2h));
  SSPCG_CUDA(cudaMemcpyAsync(status_host, status, sizeof(int32_t) * plan->nprob, cudaMemcpyDeviceToHost, plan->d2h));
  SSPCG_CUDA(cudaMemcpyAsync(relres_host, relres, sizeof(double) * plan->nprob, cudaMemcpyDeviceToHost, plan->d2h));
  SSPCG_CUDA(cudaEventRecord(a.out_done, plan->d2h));
  ++plan->acalls;
  return SSPCG_OK;
}

sspcg_status sspcg_plan_join(sspcg_plan *plan, sspcg_stream stream) {
  if (!plan) return SSPCG_ERR_INVALID_ARG;
  if (!plan->d2h) return SSPCG_OK;
  for (auto &a : plan->aslot) SSPCG_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, a.out_done, 0));
  return SSPCG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host helpers for the warm-start unit (mlp_api.cu)
// ---------------------------------------------------------------------------
namespace sspcg {
namespace host {
PlanView plan_view(const sspcg_plan *p) {
  PlanView v{};
  v.nprob = p->nprob;
  v.ps = ProbSet{p->d_desc, ProbDesc{}, p->nprob};
  v.kref = p->d_kref;
  v.knots = p->total_knots;
  v.knot_start = p->knot_start.data();
  v.d_knot_start = p->d_knot_start;
  v.total_off = p->total_off;
  v.max_nu = 0;
  for (const ProbDesc &d : p->hdesc) v.max_nu = std::max(v.max_nu, d.nu);
  return v;
}
sspcg_status build_half(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B, const float *qd,
                        const float *rd, float *D, float *E, float *PD, float *PE, int32_t *status,
                        sspcg_stream stream) {
  return pipeline_build(plan, kind, A, B, qd, rd, D, E, PD, PE, status, stream);
}
sspcg_status solve_half(sspcg_plan *plan, const float *A, const float *B, const float *qd, const float *rd,
                        const float *gamma, const float *PD, const float *PE, float *lambda, int32_t *iters,
                        double *relres, int32_t *status, int warm, sspcg_stream stream) {
  return pipeline_solve(plan, A, B, qd, rd, gamma, PD, PE, lambda, iters, relres, status, warm, stream);
}
}  // namespace host
}  // namespace sspcg
