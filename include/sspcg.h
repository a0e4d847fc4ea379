/*
 * sspcg — symmetric stair preconditioned conjugate gradient on GB300 (sm_103a).
 *
 * C ABI of the library.  It solves the Schur-complement system of the
 * equality-constrained trajectory-optimisation QP of Bu & Plancher,
 * "Symmetric Stair Preconditioning of Linear Systems for Parallel Trajectory
 * Optimization" (arXiv 2309.06427), Sec. II-A, Eq. (schur):
 *
 *     S lambda = gamma,   S = C G^-1 C^T   (block tridiagonal, SPD)
 *
 * with preconditioned CG (Sec. II-B) and the symmetric stair preconditioner
 * of Sec. IV, or the additive stair (Sec. III), block-Jacobi or Jacobi
 * preconditioners (Sec. II-C, Eq. jacobi).
 *
 * Sign convention.  The paper's S = -C G^-1 C^T is negative definite; its
 * footnote in Sec. II-A negates it.  This library works with the positive
 * definite S = C G^-1 C^T and returns mu = -lambda* of the paper.  The
 * constraint rows are -x_0 (+ x_s) and A_k x_k + B_k u_k - x_{k+1}.
 *
 * Problem data (one problem, horizon N, state size nx, input size nu),
 * FP32, row-major, contiguous:
 *   A  [N][nx][nx]   dynamics Jacobians A_k            (Sec. II-A)
 *   B  [N][nx][nu]   input Jacobians B_k
 *   qd [N+1][nx]     diagonal of the state cost Hessians Q_k (must be > 0)
 *   rd [N][nu]       diagonal of the input cost Hessians R_k (must be > 0)
 * Schur blocks, 0-based block rows k = 0..N:
 *   D  [N+1][nx][nx] D_0 = Q_0^-1,
 *                    D_k = A_{k-1} Q_{k-1}^-1 A_{k-1}^T + B_{k-1} R_{k-1}^-1 B_{k-1}^T + Q_k^-1
 *                    (= -theta_{k-1} of Sec. II-A); symmetric
 *   E  [N][nx][nx]   E[k-1] = S(k, k-1) = -A_{k-1} Q_{k-1}^-1 (= -phi_{k-1}); the
 *                    block S(k-1, k) is E[k-1]^T
 * Preconditioner blocks, same layout:
 *   PD [N+1][nx][nx] Phi^-1(k, k) = D_k^-1 (symmetric)
 *   PE [N][nx][nx]   PE[k-1] = Phi^-1(k, k-1) = -c D_k^-1 E[k-1] D_{k-1}^-1 with
 *                    c = 1 (symmetric stair, Sec. IV: Psi_l^-1 + Psi_r^-1 - D^-1),
 *                    c = 1/2 (additive stair, Sec. III), c = 0 (block-Jacobi);
 *                    Jacobi: PD_k = diag(1 / diag D_k), PE = 0.
 * Vectors gamma, lambda: [N+1][nx].
 *
 * Limits: 1 <= nx <= SSPCG_MAX_NX, 0 <= nu <= SSPCG_MAX_NX, 0 <= N <= SSPCG_MAX_N.  The
 * single-problem solves, the batched block-form solve and the allocation-free solve need
 * the PCG vectors of a problem to fit in one CTA's shared memory (about
 * 7 (N+1) nx + 2 N nu floats, at most about 56000), else they return
 * SSPCG_ERR_UNSUPPORTED; the plan-based batched QP-form calls keep such problems'
 * vectors in a plan-owned global workspace instead.
 *
 * Ownership and execution.  Every array argument is a device pointer owned
 * by the caller, 16-byte aligned, unless the parameter is documented as a
 * host pointer.  All calls are asynchronous on ``stream`` (0 = legacy
 * default stream) and return before the work is done; a returned
 * SSPCG_OK means the arguments were valid and the launches were issued.
 * Nothing is printed and nothing exits.  Per-problem outcomes (solve
 * status, iteration count, residual) are written to caller device arrays.
 * Only an sspcg_plan allocates device memory (at creation).
 */
#ifndef SSPCG_H_
#define SSPCG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CUDA stream handle (cudaStream_t), passed as an opaque pointer. */
typedef void *sspcg_stream;

#define SSPCG_MAX_NX 28
#define SSPCG_MAX_N 4096

/* Return codes of every call. */
typedef enum {
  SSPCG_OK = 0,
  SSPCG_ERR_INVALID_ARG = 1, /* null or misaligned pointer, size out of range */
  SSPCG_ERR_UNSUPPORTED = 2, /* valid request the library does not implement */
  SSPCG_ERR_CUDA = 3,        /* a CUDA runtime call failed (see sspcg_last_cuda_error) */
} sspcg_status;

/* Per-problem outcome written to the int32 ``status`` arrays. */
enum {
  SSPCG_SOLVE_OK = 0,        /* ||r||_2 <= tol * ||gamma||_2 reached */
  SSPCG_SOLVE_MAXITER = 1,   /* max_iter iterations without reaching tol */
  SSPCG_SOLVE_BREAKDOWN = 2, /* p^T S p <= 0: S not positive definite in finite precision */
  SSPCG_SOLVE_NOT_SPD = 3,   /* a diagonal block D_k failed its FP64 factorisation */
  SSPCG_SOLVE_NONFINITE = 4, /* NaN or Inf met during the iteration */
};

/* Preconditioners (Sec. II-C, III, IV). */
typedef enum {
  SSPCG_PRECOND_SYM_STAIR = 0,    /* Phi_sym^-1 = Psi_l^-1 + Psi_r^-1 - D^-1 (Sec. IV) */
  SSPCG_PRECOND_ADD_STAIR = 1,    /* Phi_add^-1 = (Psi_l^-1 + Psi_r^-1) / 2 (Sec. III) */
  SSPCG_PRECOND_BLOCK_JACOBI = 2, /* Phi = block-diag(S)  (Eq. jacobi) */
  SSPCG_PRECOND_JACOBI = 3,       /* Phi = diag(S)        (Eq. jacobi) */
} sspcg_precond;

/* Precision of the PCG dot products (p.Sp, r.z, r.r). */
enum {
  SSPCG_REDUCE_DF = 0,  /* default: exact FP32 products, double-float (~48-bit) sums */
  SSPCG_REDUCE_F32 = 1, /* FP32 products and sums (pairwise across threads) */
  SSPCG_REDUCE_F64 = 2, /* FP64 products and sums (GB300 runs FP64 at ~1/64 of FP32) */
};

/* Working precision of the batched pipeline calls (sspcg_pipeline_batched,
 * sspcg_pipeline_host, captured pipelines).  The other batched calls are FP32. */
enum {
  SSPCG_PRECISION_AUTO = 0, /* FP32; FP64 for problems of at most 192 unknowns ((N+1) nx), whose FP32
                               CG loses the finite termination the clustered spectrum gives (Thm. 4.2) */
  SSPCG_PRECISION_F32 = 1,  /* FP32 for every problem */
  SSPCG_PRECISION_F64 = 2,  /* FP64 for every problem (blocks in plan-owned FP64 memory) */
};

/* Kernel schedule of a PCG problem. */
enum {
  SSPCG_SCHED_AUTO = 0,     /* as RESIDENT */
  SSPCG_SCHED_RESIDENT = 1, /* operator and preconditioner staged once into shared memory (as many block
                               rows as fit; the rest read from L2/HBM every iteration) */
  SSPCG_SCHED_STREAM = 2,   /* operator and preconditioner read from L2/HBM every iteration */
  SSPCG_SCHED_WARP = 3,     /* plan calls: as RESIDENT, and every group of problems that fit whole in shared
                               memory (QP operator form, textbook PCG, double-float or FP64 sums) runs one
                               problem per warp, as many warps per CTA as fit (at most 16); other entry
                               points: as RESIDENT */
};

/* Solver options. */
typedef struct {
  double tol;              /* stop before an iteration once ||r||_2 <= tol * ||gamma||_2 (recurrence residual) */
  int32_t max_iter;        /* <= 0: 10 * (N + 1) * nx */
  int32_t warm_start;      /* 0: lambda_0 = 0.  1: lambda holds lambda_0 on entry.
                              2: as 1, but restart from lambda_0 = 0 when ||gamma - S lambda_0|| >= ||gamma||
                                 or lambda_0 is not finite */
  int32_t reduction;       /* SSPCG_REDUCE_* */
  int32_t schedule;        /* SSPCG_SCHED_*; RESIDENT is downgraded to STREAM for problems that do not fit */
  int32_t block_threads;   /* threads per CTA, multiple of 32 in [32, 512]; 0: chosen by the library */
  int32_t precision;       /* SSPCG_PRECISION_*: working precision of the batched pipeline calls */
  int32_t poly_degree;     /* d in [0, SSPCG_MAX_POLY_DEGREE]: the PCG applies the degree-d polynomial
                              (Neumann) preconditioner of the splitting S = Phi - (Phi - S) with Phi^-1 the
                              assembled preconditioner (Eq. polynomial_precon):
                                Phi_d^-1 = sum_{j=0..d} (I - Phi^-1 S)^j Phi^-1.
                              d = 0 is Phi^-1 itself.  Applied as z <- z + Phi^-1 (r - S z), d times after
                              z = Phi^-1 r: d more products with S and with Phi^-1 per iteration, one more
                              vector of shared memory.  Symmetric for every d; positive definite when the
                              splitting converges (rho(I - Phi^-1 S) < 1, true for the symmetric stair, the
                              additive stair and block-Jacobi; for scalar Jacobi only when 2 diag(S) - S is
                              positive definite), and then eig(Phi_d^-1 S) = 1 - (1 - theta)^(d+1) for the
                              eigenvalues theta of Phi^-1 S.  On the symmetric stair, degree d equals degree
                              2d+1 on the block-Jacobi splitting. */
  int32_t cg_variant;      /* 0: textbook PCG (Saad Alg. 9.1).  1: single-reduction PCG (Chronopoulos and
                              Gear 1989): the same iterates in exact arithmetic, s = S p kept by recurrence,
                              and (r.u, S u.u, r.r) in one block sum per iteration (one barrier and one
                              reduction tree fewer).  Run by the QP-form FP32 solves; requires
                              SSPCG_REDUCE_DF (SSPCG_ERR_INVALID_ARG otherwise); the FP64 and block-form
                              solves stay textbook.  With poly_degree d > 0, u = Phi_d^-1 r as above.  With
                              block-Jacobi blocks, d = 1 and no PE this applies the symmetric stair
                              implicitly, Phi_sym^-1 = 2 D^-1 - D^-1 S D^-1 (Sec. IV with Eq. stair_inv), with
                              one reduction per iteration.  iters counts x updates either way. */
} sspcg_options;

#define SSPCG_MAX_POLY_DEGREE 16

/* Message of the last CUDA error seen by this thread (static storage, never NULL). */
const char *sspcg_last_cuda_error(void);

/* Library version string. */
const char *sspcg_version(void);

/*
 * Diagnostic (no counterpart in the paper): measured shared-memory read
 * bandwidth of the current device, the peak the PCG kernel's roofline is
 * reported against.  Two 1024-thread CTAs per SM read a 48 KB shared buffer
 * ``rounds`` times with conflict-free loads of ``load_bytes`` (4 or 16)
 * bytes; *gbytes_per_s = bytes read / kernel time (CUDA events, after one
 * warm-up launch).  Synchronises ``stream``; allocates a small device buffer.
 * Errors: SSPCG_ERR_INVALID_ARG for other sizes or rounds <= 0.
 */
sspcg_status sspcg_measure_smem_bandwidth(int32_t load_bytes, int32_t rounds, double *gbytes_per_s,
                                          sspcg_stream stream);

/* ------------------------------------------------------------------ */
/* Single problem                                                     */
/* ------------------------------------------------------------------ */

/*
 * Schur blocks D, E from the QP data (Sec. II-A, the theta_k/phi_k block
 * formulas, negated).  FP32 arithmetic; D_k is written exactly symmetric.
 * Inputs A, B, qd, rd; outputs D [N+1][nx][nx], E [N][nx][nx].
 */
sspcg_status sspcg_build_schur(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                               const float *rd, float *D, float *E, sspcg_stream stream);

/*
 * Preconditioner blocks PD, PE from D, E (Eq. stair_inv with Sec. III/IV, or
 * Eq. jacobi).  D_k^-1 is formed by an FP64 LDL^T factorisation of each
 * diagonal block; the off-diagonal products -c D_k^-1 E D_{k-1}^-1 run in FP32.
 * ``status`` (device, 1 int32) is set to SSPCG_SOLVE_OK, or to
 * SSPCG_SOLVE_NOT_SPD when some D_k is not positive definite.
 */
sspcg_status sspcg_build_precond(int32_t N, int32_t nx, sspcg_precond kind, const float *D, const float *E, float *PD,
                                 float *PE, int32_t *status, sspcg_stream stream);

/*
 * PCG on S lambda = gamma with S given by its blocks D, E (Sec. II-B) and
 * Phi^-1 by PD, PE.  One CTA solves the problem: matrix-vector products in
 * FP32, dot products in the precision opts->reduction selects.
 * ``lambda`` is the solution (and lambda_0 on entry when opts->warm_start).
 * Outputs (device, 1 element each): iters = number of S*p products,
 * relres = ||r||_2 / ||gamma||_2 of the recurrence residual, status.
 * gamma = 0 gives lambda = 0, iters = 0.
 * PE may be NULL: the preconditioner is then block-diagonal (block-Jacobi,
 * or Jacobi's diagonal blocks), and its off-diagonal blocks are neither
 * staged nor read; the same holds for every solve entry point below and for
 * the pipelines with SSPCG_PRECOND_BLOCK_JACOBI or SSPCG_PRECOND_JACOBI,
 * which pass no PE to their solves.
 */
sspcg_status sspcg_solve(int32_t N, int32_t nx, const float *D, const float *E, const float *PD, const float *PE,
                         const float *gamma, float *lambda, const sspcg_options *opts, int32_t *iters,
                         double *relres, int32_t *status, sspcg_stream stream);

/*
 * As sspcg_solve, but S is applied in the factored form of its definition,
 * S p = C (G^-1 (C^T p)) (Eq. schur), from the QP data A, B, qd, rd.  The
 * FP32 inputs are then the operator itself: no rounding of S's blocks enters
 * the system, which keeps lambda within 1e-5 of the FP64 solution on
 * ill-conditioned systems where FP32 blocks of S do not.
 */
sspcg_status sspcg_solve_qp(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                            const float *rd, const float *PD, const float *PE, const float *gamma, float *lambda,
                            const sspcg_options *opts, int32_t *iters, double *relres, int32_t *status,
                            sspcg_stream stream);

/*
 * FP64 path of the same three steps (the working precision of blocks,
 * vectors and lambda is double; inputs stay FP32 and convert exactly).  For
 * problems whose FP64 iteration count must be reproduced: FP32 rounding of
 * Phi^-1 or of the vectors splits the doubled eigenvalue clusters of
 * Thm. 4.2 by ~1e-7 and delays CG's finite termination (e.g. 21 -> 25..42
 * iterations on nx = 2, N = 20).  FP64 runs at about 1/64 of the FP32 rate
 * on GB300, so this path suits small problems.
 */
sspcg_status sspcg_build_schur_f64(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B,
                                   const float *qd, const float *rd, double *D, double *E, sspcg_stream stream);
sspcg_status sspcg_build_precond_f64(int32_t N, int32_t nx, sspcg_precond kind, const double *D, const double *E,
                                     double *PD, double *PE, int32_t *status, sspcg_stream stream);
sspcg_status sspcg_solve_qp_f64(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                                const float *rd, const double *PD, const double *PE, const float *gamma,
                                double *lambda, const sspcg_options *opts, int32_t *iters, double *relres,
                                int32_t *status, sspcg_stream stream);

/*
 * True residual ||gamma - S lambda||_2 / ||gamma||_2 with S = C G^-1 C^T
 * applied in FP64 from the QP data (diagnostic).  relres_true: device, 1 double.
 */
sspcg_status sspcg_residual_qp(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                               const float *rd, const float *gamma, const float *lambda, double *relres_true,
                               sspcg_stream stream);

/* ------------------------------------------------------------------ */
/* Batches of independent problems of uneven N, nx, nu                */
/* ------------------------------------------------------------------ */

/*
 * A plan describes a batch.  Problem i's arrays are packed back to back in
 * one device buffer per array kind, each problem starting at a 16-byte
 * aligned offset given by sspcg_plan_offsets.  The plan owns its device
 * descriptors and work lists (allocated here, freed by sspcg_plan_destroy)
 * and picks a kernel schedule per problem class.  It also holds padded
 * copies of A, B and PE for the problems that do not fit in shared memory
 * whole (every problem under SSPCG_SCHED_STREAM): about N nx (2 nx4 + nu4) floats
 * each, with nx4 and nu4 rounded up to multiples of 4.  The QP-form batched
 * solves rewrite them from their arguments on every call, and the PCG reads
 * the streamed block rows from them with 128-bit loads.
 * N, nx, nu: host arrays of nprob entries.  opts: host pointer, copied.
 */
typedef struct sspcg_plan sspcg_plan;

/* Packed array kinds. */
typedef enum {
  SSPCG_ARRAY_A = 0,    /* N*nx*nx per problem */
  SSPCG_ARRAY_B = 1,    /* N*nx*nu */
  SSPCG_ARRAY_QD = 2,   /* (N+1)*nx */
  SSPCG_ARRAY_RD = 3,   /* N*nu */
  SSPCG_ARRAY_DIAG = 4, /* (N+1)*nx*nx: D and PD */
  SSPCG_ARRAY_OFF = 5,  /* N*nx*nx: E and PE */
  SSPCG_ARRAY_VEC = 6,  /* (N+1)*nx: gamma and lambda */
  SSPCG_ARRAY_RFULL = 7, /* N*nu*nu: full R_k blocks (sspcg_build_schur_full_batched) */
  SSPCG_NUM_ARRAYS = 8
} sspcg_array;

sspcg_status sspcg_plan_create(sspcg_plan **plan, int32_t nprob, const int32_t *N, const int32_t *nx,
                               const int32_t *nu, const sspcg_options *opts);
sspcg_status sspcg_plan_destroy(sspcg_plan *plan);

/* Total floats of each packed array kind (host out[SSPCG_NUM_ARRAYS]). */
sspcg_status sspcg_plan_sizes(const sspcg_plan *plan, int64_t *out);

/* Float offset of each problem in a packed array kind (host out[nprob]). */
sspcg_status sspcg_plan_offsets(const sspcg_plan *plan, sspcg_array kind, int64_t *out);

/*
 * Schedule summary (host out[8]): [0] PCG launches of a pipeline call, [1]
 * FP32 problems staged in shared memory, [2] FP32 problems streamed from
 * L2/HBM, [3] FP64 problems, [4] PCG launches of sspcg_solve_qp_batched,
 * [5] of sspcg_solve_batched, [6]/[7] resident/streamed problems of
 * sspcg_solve_qp_batched.
 */
sspcg_status sspcg_plan_stats(const sspcg_plan *plan, int64_t *out);

/*
 * Phase timing.  When enabled, the plan records CUDA events on the call's
 * stream around the preconditioner build and the PCG launches of each
 * pipeline or solve call; sspcg_plan_timings waits for the last call and
 * returns out_ms[0] = build time (0 for solve-only calls), out_ms[1] = PCG
 * time.  Disabled while capturing a graph.
 */
sspcg_status sspcg_plan_set_timing(sspcg_plan *plan, int32_t enable);
sspcg_status sspcg_plan_timings(sspcg_plan *plan, float *out_ms);

/* Batched sspcg_build_schur over packed arrays. */
sspcg_status sspcg_build_schur_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                       const float *rd, float *D, float *E, sspcg_stream stream);

/*
 * Schur blocks with full SPD cost blocks (Sec. II-A, where the block formulas
 * carry Q_k^-1 and R_k^-1 as matrices):
 *   D_0 = Q_0^-1,  D_{k+1} = A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T + Q_{k+1}^-1,
 *   E_k = S(k+1, k) = -A_k Q_k^-1.
 * Q: FP32 [N+1][nx][nx], R: FP32 [N][nu][nu], row-major and symmetric (only
 * the lower triangles are read).  Q_k^-1 and R_k^-1 are formed by FP64 LDL^T
 * (as the D_k^-1 of sspcg_build_precond) and rounded to FP32 once; the products
 * are FP32, D_k exactly symmetric.  The result feeds sspcg_build_precond and
 * the block-form solves (sspcg_solve, sspcg_solve_batched); the QP-form calls
 * take diagonal Q and R only.
 * status (device int32, one per problem): 0, or SSPCG_SOLVE_NOT_SPD when a Q_k or
 * R_k is not positive definite (that inverse is set to zero, so D and E are
 * then meaningless).  The preconditioner build resets status: read it first.
 * Single problem: work is caller-owned device scratch of
 * sspcg_schur_full_work_floats(N, nx, nu) floats, 16-byte aligned.
 * Batched: Q packed like D (SSPCG_ARRAY_DIAG), R in SSPCG_ARRAY_RFULL; the
 * plan allocates its scratch on first use.
 */
sspcg_status sspcg_schur_full_work_floats(int32_t N, int32_t nx, int32_t nu, int64_t *floats);
sspcg_status sspcg_build_schur_full(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *Q,
                                    const float *R, float *D, float *E, float *work, int32_t *status,
                                    sspcg_stream stream);
sspcg_status sspcg_build_schur_full_batched(sspcg_plan *plan, const float *A, const float *B, const float *Q,
                                            const float *R, float *D, float *E, int32_t *status,
                                            sspcg_stream stream);

/* Batched sspcg_build_precond; status: device int32[nprob]. */
sspcg_status sspcg_build_precond_batched(sspcg_plan *plan, sspcg_precond kind, const float *D, const float *E,
                                         float *PD, float *PE, int32_t *status, sspcg_stream stream);

/* Batched sspcg_solve (block S). iters, status: int32[nprob]; relres: double[nprob].
 * SSPCG_ERR_UNSUPPORTED when a problem's PCG vectors (about 7 (N+1) nx values) exceed one CTA's shared
 * memory: the block form has no global-workspace kernels (the QP-form calls do). */
sspcg_status sspcg_solve_batched(sspcg_plan *plan, const float *D, const float *E, const float *PD,
                                 const float *PE, const float *gamma, float *lambda, int32_t *iters,
                                 double *relres, int32_t *status, sspcg_stream stream);

/* Batched sspcg_solve_qp (factored S). */
sspcg_status sspcg_solve_qp_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                    const float *rd, const float *PD, const float *PE, const float *gamma,
                                    float *lambda, int32_t *iters, double *relres, int32_t *status,
                                    sspcg_stream stream);

/* Batched sspcg_residual_qp; relres_true: double[nprob]. */
sspcg_status sspcg_residual_qp_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                       const float *rd, const float *gamma, const float *lambda,
                                       double *relres_true, sspcg_stream stream);

/*
 * The whole path for a batch, from QP data to lambda: Schur blocks,
 * preconditioner, PCG with the factored S.  D, E, PD, PE are caller work
 * buffers of the packed sizes.  A problem whose preconditioner fails keeps
 * status SSPCG_SOLVE_NOT_SPD and is not iterated.
 * Schedule: every problem's blocks are built first (FP32, and FP64 for the
 * FP64 subset the plan's precision option selects); then all PCG launch
 * groups run concurrently on plan-owned streams forked from ``stream``,
 * the group with the most estimated work first, and join back into it.
 * Capturable as a CUDA graph (sspcg_plan_capture_pipeline).
 */
sspcg_status sspcg_pipeline_batched(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                    const float *qd, const float *rd, const float *gamma, float *D, float *E,
                                    float *PD, float *PE, float *lambda, int32_t *iters, double *relres,
                                    int32_t *status, sspcg_stream stream);

/*
 * Capture sspcg_pipeline_batched with these pointers into a CUDA graph owned
 * by the plan (the call first runs the pipeline once uncaptured); then
 * sspcg_plan_launch replays it.  ``stream`` must not be the legacy default
 * stream.  A later capture replaces the graph.
 */
sspcg_status sspcg_plan_capture_pipeline(sspcg_plan *plan, sspcg_precond kind, const float *A, const float *B,
                                         const float *qd, const float *rd, const float *gamma, float *D, float *E,
                                         float *PD, float *PE, float *lambda, int32_t *iters, double *relres,
                                         int32_t *status, sspcg_stream stream);
sspcg_status sspcg_plan_launch(sspcg_plan *plan, sspcg_stream stream);

/*
 * Autotuner (the batched schedule of Sec. II-B's PCG; the paper fixes no
 * parallel schedule).  Builds the blocks and preconditioner like
 * sspcg_pipeline_batched, then, for every PCG launch group of the chosen
 * sets (which: SSPCG_TUNE_PIPELINE, the pipeline's FP32 and FP64 sets;
 * SSPCG_TUNE_SOLVE, the set of sspcg_solve_qp_batched; or both; one group
 * per nx and residency class), times candidate schedules alone on these
 * inputs: block sizes 64..512 threads (16 rows per thread to one); for
 * groups that do not fit in shared memory whole, staging the first rows into
 * the whole budget or into 1/2, 1/3 or 1/4 of it (several CTAs per SM), or
 * streaming every block row from L2; for groups that do fit (QP form,
 * textbook PCG, double-float or FP64 sums), also one problem per warp with
 * 1 to 16 warps per CTA.  Each group keeps its fastest
 * candidate (grid from the kernel's occupancy at that block size); the
 * choices also go to a process-wide cache keyed by (launch set, operator form,
 * precision, reduction, polynomial degree, PCG variant, nx, residency class,
 * bucket of the largest N: <16, <32, ..., <512, >=512), which later
 * sspcg_plan_create calls with block_threads = 0 and the automatic schedule
 * apply to matching groups.  Costs about 30 launches of each group.
 * Arguments as sspcg_pipeline_batched; lambda, iters and relres are
 * overwritten (a warm start is not used while tuning); status holds the
 * preconditioner's codes afterwards.  A captured pipeline graph is dropped
 * (capture again).  Synchronises ``stream``.
 */
#define SSPCG_TUNE_PIPELINE 1
#define SSPCG_TUNE_SOLVE 2
sspcg_status sspcg_plan_autotune(sspcg_plan *plan, int32_t which, sspcg_precond kind, const float *A, const float *B,
                                 const float *qd, const float *rd, const float *gamma, float *D, float *E, float *PD,
                                 float *PE, float *lambda, int32_t *iters, double *relres, int32_t *status,
                                 sspcg_stream stream);

/* Fields per group of sspcg_plan_schedule. */
#define SSPCG_SCHEDULE_FIELDS 11
/*
 * The PCG launch groups of a plan: which = 0 (the pipeline's FP32 set),
 * 1 (its FP64 set), 2 (sspcg_solve_qp_batched).  *count = number of groups;
 * the first min(capacity, count) rows of SSPCG_SCHEDULE_FIELDS int32 go to
 * out: nx, residency class (0 partially staged, 1..4 fully staged, 5
 * vectors in global memory), problems, largest N, block threads, grid CTAs,
 * dynamic shared memory bytes, streams every block row (0/1), chosen by the
 * tuner or its cache (0/1), shared-memory share (a partially staged group
 * stages into 1/share of the budget, so up to share CTAs fit on an SM),
 * warps per CTA when each warp solves its own problem (0: one problem per
 * CTA).
 */
sspcg_status sspcg_plan_schedule(const sspcg_plan *plan, int32_t which, int32_t *out, int32_t capacity,
                                 int32_t *count);
/* Forget every cached tuning choice. */
sspcg_status sspcg_autotune_cache_clear(void);

/*
 * sspcg_pipeline_batched from HOST buffers (packed like the device arrays):
 * copies the inputs to plan-owned device buffers (allocated on first use),
 * runs the path, copies lambda, iters, relres and status back and waits for
 * the stream.  Host buffers should be pinned for full copy speed.  With
 * warm_start set in the plan's options, lambda_host holds lambda_0 on entry.
 */
sspcg_status sspcg_pipeline_host(sspcg_plan *plan, sspcg_precond kind, const float *A_host, const float *B_host,
                                 const float *qd_host, const float *rd_host, const float *gamma_host,
                                 float *lambda_host, int32_t *iters_host, double *relres_host, int32_t *status_host,
                                 sspcg_stream stream);

/*
 * sspcg_pipeline_host without the final wait: call i copies its inputs into
 * plan-owned device slot i % 2 on a plan copy stream, runs the path on
 * ``stream``, and copies the results to the host buffers on a second plan
 * copy stream, so that one call's copies overlap the previous call's
 * compute.  Computes of successive calls run in call order even on
 * different streams.  The host buffers should be pinned (pageable ones
 * work but serialise the copies) and stay untouched until the results are
 * complete: after sspcg_plan_join(plan, s) once stream s has completed.
 * Inputs are only read, so calls may share them; with options.warm_start
 * lambda_host is read as the starting point when the call's copies run,
 * which is not ordered after an earlier in-flight call's copy-out, so a
 * warm-started call that must start from the previous result joins first.
 * Allocates on first use two slots of inputs and outputs and one set of
 * D, E, PD, PE blocks, kept until sspcg_plan_destroy.
 */
sspcg_status sspcg_pipeline_host_async(sspcg_plan *plan, sspcg_precond kind, const float *A_host,
                                       const float *B_host, const float *qd_host, const float *rd_host,
                                       const float *gamma_host, float *lambda_host, int32_t *iters_host,
                                       double *relres_host, int32_t *status_host, sspcg_stream stream);
/* Make ``stream`` wait for every copy of the plan's earlier asynchronous host pipeline calls. */
sspcg_status sspcg_plan_join(sspcg_plan *plan, sspcg_stream stream);

/* ------------------------------------------------------------------ */
/* Batched solve without allocation                                   */
/* ------------------------------------------------------------------ */

/* Largest batch of sspcg_solve_qp_batched_noalloc. */
#define SSPCG_NOALLOC_MAX_PROBLEMS 4096

/*
 * sspcg_solve_qp_batched without a plan and without allocating anything,
 * for callers that cannot call cudaMalloc once running: a model-predictive
 * control loop on a real-time thread (cudaMalloc may synchronise the device
 * and take unbounded time), or an application whose own allocator owns all
 * device memory.  The paper has no counterpart; this is a library service.
 *
 * N, nx, nu: HOST arrays of nprob <= SSPCG_NOALLOC_MAX_PROBLEMS entries;
 * more return SSPCG_ERR_INVALID_ARG.  The device arrays are packed as by a
 * plan (sspcg_plan_offsets): problem i of each array kind starts at the
 * prefix sum of the sizes of problems 0..i-1, each size rounded up to a
 * multiple of 4 elements.  Other arguments as in sspcg_solve_qp_batched
 * (FP32, factored S).
 *
 * Scratch: problem descriptors, the work list and work-queue counters live
 * in one file-scope __device__ array of 311,552 bytes (4096 descriptors),
 * which every GPU that loads the library holds until the process exits.
 * All calls share the array, so calls that overlap on the GPU (on different
 * streams without ordering) race and give wrong results.  No cudaMalloc,
 * cudaFree or allocating library routine is called, and no host heap is
 * used (about 25 KB of the calling thread's stack).
 *
 * Host behaviour: the call copies nothing with cudaMemcpy.  The shapes and
 * the work order travel as the parameter block of one set-up kernel (the
 * driver copies launch parameters when it records the launch), which writes
 * the descriptors into the array and clears the queue counters and
 * ``status`` on ``stream``; then one PCG launch per nx follows.  The call
 * returns without waiting for the GPU.
 *
 * Warm-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make it before any stream capture.  Later calls
 * can be captured into a CUDA graph: they launch kernels only, so a replay
 * solves the captured batch again (same shapes and pointers).  The first
 * launch of each PCG kernel variant (each nx and each reduction, schedule or
 * CG option) sets that kernel's shared-memory attribute and, under lazy
 * module loading, may load its code.  Callers with a time bound (a control
 * loop) should make one call per nx and option set they will use before the
 * loop starts; later calls do neither.
 */
sspcg_status sspcg_solve_qp_batched_noalloc(int32_t nprob, const int32_t *N, const int32_t *nx, const int32_t *nu,
                                            const float *A, const float *B, const float *qd, const float *rd,
                                            const float *PD, const float *PE, const float *gamma, float *lambda,
                                            const sspcg_options *opts, int32_t *iters, double *relres,
                                            int32_t *status, sspcg_stream stream);

/* ------------------------------------------------------------------ */
/* Learned warm start                                                 */
/* ------------------------------------------------------------------ */
/*
 * A 3-layer ReLU network maps the data of each knot to an initial guess
 * lambda_0 for the PCG solve.  The paper has no learned component: this is
 * the warm-start extension of the method (a plain start lambda_0 = 0 remains
 * the fallback, sspcg_options.warm_start = 2).
 *
 * Knot features: row k of a problem (one per block row of S) holds, as FP32
 * values normalised per column and rounded to bfloat16, in 1344 columns:
 *   [0, 784)      A_{k-1} as [28][28] row-major (zero padded; zero for k = 0)
 *   [784, 1176)   B_{k-1} as [28][14] row-major (zero padded; zero for k = 0)
 *   [1176, 1204)  diag Q_{k-1}   [1204, 1218) diag R_{k-1}   (zero for k = 0)
 *   [1218, 1246)  diag Q_k       [1246, 1274) gamma_k
 *   [1274, 1302)  D_k^-1 gamma_k (from the preconditioner's diagonal blocks PD)
 *   1302          nx / 28        [1303, 1344) zero
 * These are the data from which block row k of S is built (Sec. II-A).
 * Normalisation: x -> (x - mu) * inv_sigma per column.
 *
 * Network: H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3;
 * lambda_0 of knot k = Y[k][0..nx).  Parameters are FP32 masters, flat in the
 * order W1 [256][1344], b1 [256], W2 [256][256], b2 [256], W3 [32][256],
 * b3 [32] (SSPCG_MLP_PARAMS floats); the products use bfloat16 copies of the
 * weights and of X, H1, H2 and the output gradient, with FP32 accumulation.
 *
 * Training loss of a minibatch of P whole problems: the mean over problems
 * of ||S (lambda_0 - lambda*)||^2 / ||gamma||^2, where lambda* is the plain
 * method's solution.  Since S lambda* = gamma up to the solve tolerance this
 * is the squared relative initial residual that the PCG exit test measures.
 * Optimiser: Adam (Kingma & Ba 2015) on the FP32 masters.
 *
 * The problem tables (shapes, packed offsets) come from a plan; every array
 * argument is a device pointer in the plan's packed layout.  A network object
 * owns its parameters, Adam state and the workspace of max_rows knot rows.
 * The layout holds nu <= 14: calls on a plan with a larger nu return
 * SSPCG_ERR_UNSUPPORTED.
 */
#define SSPCG_MLP_IN 1344
#define SSPCG_MLP_HIDDEN 256
#define SSPCG_MLP_OUT 32
#define SSPCG_MLP_PARAMS 418336

typedef struct sspcg_mlp sspcg_mlp;

typedef struct {
  float lr;    /* step size */
  float beta1; /* first-moment decay */
  float beta2; /* second-moment decay */
  float eps;   /* denominator guard */
} sspcg_adam;

/* Engines of the forward products (inference and the training forward pass; the backward products
 * always use mma.sync):
 *   SSPCG_MLP_ENGINE_TCGEN05  tcgen05.mma with TMEM accumulators, operands staged by TMA (default)
 *   SSPCG_MLP_ENGINE_MMA_SYNC mma.sync.m16n8k16 with register accumulators */
enum { SSPCG_MLP_ENGINE_TCGEN05 = 0, SSPCG_MLP_ENGINE_MMA_SYNC = 1 };

/* Create a network with workspace for max_rows >= 1 knot rows per call chunk.
 * Parameters start at zero; normalisation at mu = 0, inv_sigma = 1. */
sspcg_status sspcg_mlp_create(sspcg_mlp **mlp, int32_t max_rows);
sspcg_status sspcg_mlp_destroy(sspcg_mlp *mlp);
/* Select the forward-product engine; SSPCG_ERR_UNSUPPORTED when TMA descriptors cannot be made. */
sspcg_status sspcg_mlp_set_engine(sspcg_mlp *mlp, int32_t engine);
/* Synchronous: *flag = 1 if a tensor-core product gave up on a bounded wait since creation, else 0. */
sspcg_status sspcg_mlp_status(const sspcg_mlp *mlp, int32_t *flag);
/* Copy SSPCG_MLP_PARAMS FP32 values from a device array into the network and reset the Adam state. */
sspcg_status sspcg_mlp_set_params(sspcg_mlp *mlp, const float *params, sspcg_stream stream);
/* Copy the FP32 parameters (or the gradients of the last training step) to a device array. */
sspcg_status sspcg_mlp_get_params(const sspcg_mlp *mlp, float *params, sspcg_stream stream);
sspcg_status sspcg_mlp_get_grads(const sspcg_mlp *mlp, float *grads, sspcg_stream stream);

/*
 * Checkpoint of a network for bit-exact resumption of training (no
 * counterpart in the paper; the warm start is this library's addition):
 * the FP32 parameters (masters), Adam's first and second moments, the Adam
 * step count and the feature normalisation, in a versioned blob in HOST
 * memory of sspcg_mlp_checkpoint_bytes() bytes, owned by the caller.  The
 * bf16 weight copies are derived from the masters on load.  Both calls
 * synchronise ``stream``.  Resuming from a checkpoint on the same GPU gives
 * the same parameters, bit for bit, as training without the interruption.
 * Errors: SSPCG_ERR_INVALID_ARG for a short buffer, or on load for a blob
 * whose magic, version or layer sizes differ.
 */
sspcg_status sspcg_mlp_checkpoint_bytes(int64_t *bytes);
sspcg_status sspcg_mlp_save(const sspcg_mlp *mlp, void *host_buf, int64_t bytes, sspcg_stream stream);
sspcg_status sspcg_mlp_load(sspcg_mlp *mlp, const void *host_buf, int64_t bytes, sspcg_stream stream);
/* Per-column normalisation (device arrays of SSPCG_MLP_IN floats). */
sspcg_status sspcg_mlp_set_normalisation(sspcg_mlp *mlp, const float *mu, const float *inv_sigma,
                                         sspcg_stream stream);
sspcg_status sspcg_mlp_get_normalisation(const sspcg_mlp *mlp, float *mu, float *inv_sigma, sspcg_stream stream);
/* Fit the normalisation to every knot of the plan's batch: mu = column mean, inv_sigma = 1 / population
 * standard deviation (FP64 sums); a column whose standard deviation is at most 1e-6 of its RMS is constant
 * and gets inv_sigma = 0.  PD: diagonal preconditioner blocks D_k^-1 (any block preconditioner). */
sspcg_status sspcg_mlp_fit_normalisation(sspcg_mlp *mlp, const sspcg_plan *plan, const float *A, const float *B,
                                         const float *qd, const float *rd, const float *gamma, const float *PD,
                                         sspcg_stream stream);
/* Normalised bfloat16 feature rows of problems [p_begin, p_end) into X [rows][SSPCG_MLP_IN] (uint16 bit
 * patterns), rows in problem order.  The rows must fit the network's max_rows. */
sspcg_status sspcg_mlp_features(const sspcg_mlp *mlp, const sspcg_plan *plan, int32_t p_begin, int32_t p_end,
                                const float *A, const float *B, const float *qd, const float *rd,
                                const float *gamma, const float *PD, uint16_t *X, sspcg_stream stream);
/* lambda_0 for every problem of the plan, written into lambda0 (vector layout). */
sspcg_status sspcg_mlp_infer(sspcg_mlp *mlp, const sspcg_plan *plan, const float *A, const float *B,
                             const float *qd, const float *rd, const float *gamma, const float *PD, float *lambda0,
                             sspcg_stream stream);
/* One training step on problems [p_begin, p_end) (whole problems; their rows must fit max_rows): forward,
 * loss, backward and one Adam step.  D, E: FP32 Schur blocks (sspcg_build_schur_batched); PD: D_k^-1 blocks;
 * lambda_star: the plain method's solutions (vector layout).  loss: device FP64 scalar (the minibatch loss
 * before the update). */
sspcg_status sspcg_mlp_train_step(sspcg_mlp *mlp, const sspcg_plan *plan, int32_t p_begin, int32_t p_end,
                                  const float *A, const float *B, const float *qd, const float *rd,
                                  const float *gamma, const float *D, const float *E, const float *PD,
                                  const float *lambda_star, const sspcg_adam *hyper, double *loss,
                                  sspcg_stream stream);
/* sspcg_pipeline_batched started from the network's lambda_0: blocks and preconditioner, inference into
 * lambda, then PCG with warm start and fallback to lambda_0 = 0 (warm_start = 2) for every problem. */
sspcg_status sspcg_pipeline_warm_batched(sspcg_plan *plan, sspcg_mlp *mlp, sspcg_precond kind, const float *A,
                                         const float *B, const float *qd, const float *rd, const float *gamma,
                                         float *D, float *E, float *PD, float *PE, float *lambda, int32_t *iters,
                                         double *relres, int32_t *status, sspcg_stream stream);

/* ------------------------------------------------------------------ */
/* The QP step around the solve (Eq. schur)                           */
/* ------------------------------------------------------------------ */
/*
 * The paper's Eq. (schur) is self-consistent for the QP of minimising
 * z^T G z / 2 - g^T z subject to C z = c, whose step is found by
 *   gamma = c - C G^-1 g,  S lambda* = gamma (S = -C G^-1 C^T),  delta z = G^-1 (g - C^T lambda*).
 * The library solves (C G^-1 C^T) mu = gamma, mu = -lambda* (see the sign note above), so
 *   delta z = G^-1 (g + C^T mu).
 * g = (q_0, r_0, q_1, ..., q_N) is the cost gradient; c [N+1][nx] holds the
 * constraint values (row 0: initial state, row k+1: dynamics defect of knot k).
 * In the block notation of Sec. II-A (zeta_k = A_k Q_k^-1 q_k + B_k R_k^-1 r_k - Q_{k+1}^-1 q_{k+1}):
 *   gamma_0 = c_0 + Q_0^-1 q_0,  gamma_{k+1} = c_{k+1} - zeta_k.
 * (The paper's block listing writes c + zeta_k; Eq. (schur)'s sign is used.)
 * Layouts: c, q, gamma, mu, dx like gamma ([N+1][nx]); r, du like diag R ([N][nu]).
 * FP32 in and out; one pass over A and B.
 */
sspcg_status sspcg_form_gamma(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                              const float *rd, const float *c, const float *q, const float *r, float *gamma,
                              sspcg_stream stream);
sspcg_status sspcg_recover_step(int32_t N, int32_t nx, int32_t nu, const float *A, const float *B, const float *qd,
                                const float *rd, const float *q, const float *r, const float *mu, float *dx,
                                float *du, sspcg_stream stream);
/* The same over a plan's packed arrays (c, q, gamma, mu, dx: SSPCG_ARRAY_VEC; r, du: SSPCG_ARRAY_RD). */
sspcg_status sspcg_form_gamma_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                      const float *rd, const float *c, const float *q, const float *r, float *gamma,
                                      sspcg_stream stream);
sspcg_status sspcg_recover_step_batched(sspcg_plan *plan, const float *A, const float *B, const float *qd,
                                        const float *rd, const float *q, const float *r, const float *mu, float *dx,
                                        float *du, sspcg_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SSPCG_H_ */
