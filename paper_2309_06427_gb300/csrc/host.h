// Host helpers defined in api.cu for the other entry-point units.
#pragma once

#include <cstdint>

#include "../../include/sspcg.h"
#include "common.cuh"

namespace sspcg {
namespace host {

// Read-only view of a plan's problem tables.
struct PlanView {
  int32_t nprob;
  ProbSet ps;                   // device descriptors
  const int2 *kref;             // (problem, block row) per knot, problems in order
  int64_t knots;                // number of knots (rows of kref)
  const int64_t *knot_start;    // host: first knot of each problem, nprob + 1 entries
  const int64_t *d_knot_start;  // the same on the device
  int64_t total_off;            // number of off-diagonal blocks
  int32_t max_nu;               // largest nu of the batch
};

int sms();
sspcg_status cuda_error(cudaError_t e);
PlanView plan_view(const sspcg_plan *p);
// The two halves of sspcg_pipeline_batched: blocks and preconditioner, then the PCG launches
// (``warm`` overrides the plan's warm-start option).
sspcg_status build_half(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B, const float *qd,
                        const float *rd, float *D, float *E, float *PD, float *PE, int32_t *status,
                        sspcg_stream stream);
sspcg_status solve_half(sspcg_plan *plan, const float *A, const float *B, const float *qd, const float *rd,
                        const float *gamma, const float *PD, const float *PE, float *lambda, int32_t *iters,
                        double *relres, int32_t *status, int warm, sspcg_stream stream);

}  // namespace host
}  // namespace sspcg
