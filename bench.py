"""Benchmark: batched symmetric-stair PCG solves/s on the ragged 4096-problem workload.

One step = the whole path over one batch, inputs resident in HBM: Schur blocks -> symmetric stair
preconditioner -> PCG to relative residual 1e-6, as one CUDA graph (sspcg_plan_launch of the pipeline
captured after sspcg_plan_autotune picked every launch group's schedule).  Prints one JSON line (rank 0)
with the phase rooflines, the end-to-end figure through the host-buffer entry point, the reduction-precision
and warm-start comparisons, the MPC workload (16,384 problems, 10 re-solves: plain, previous-solution and
learned warm starts) and the FP64 oracle on the host cores, whose solutions of sampled problems also give
the lambda error of every GPU result.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle (the reference arm) on the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_06427_gb300 import problems as P  # noqa: E402

METRIC = "PCG solves/s at rel-resid 1e-6 (batched+warm-start vs plain); iters; % BW peak"
UNIT = "solves/s"
WORKLOAD = P.RAGGED_BATCH_4096
PRECOND = "sym"
SMEM_BYTES_PER_CLK_PER_SM = 128  # shared-memory bandwidth of one SM (32 banks x 4 B per clock)
MLP_FLOP_PER_ROW = 2 * (1344 * 256 + 256 * 256 + 256 * 32)  # warm-start network forward, one knot row
def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the PCG kernel source (pcg.cuh, and its layout and arguments in
    kernels.h) with comments and blank space removed, so that only code changes alter it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("pcg.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_2309_06427_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


TRAFFIC_FILE = "pcg_kernel_traffic.md"


def pcg_traffic():
    """DRAM bytes per PCG launch set of the benchmark batch, from the committed ncu summary TRAFFIC_FILE under
    profiles/, if the kernel source is unchanged since it was captured (kernel_source_hash); else None."""
    try:
        text = open(os.path.join(ROOT, "profiles", TRAFFIC_FILE)).read()
        vals = dict(line.split(":", 1) for line in text.splitlines()
                    if line.startswith(("pcg_traffic_bytes_per_launch:", "source_sha256_16:")))
        if kernel_source_hash() != vals["source_sha256_16"].strip():
            return None
        return int(vals["pcg_traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _hbm_peak():
    """Measured HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json beside this file, else 6800 (fallback)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()


def _bf16_peak():
    """Measured dense bf16 burst throughput (TFLOP/s) from MEASURED_PEAKS.json, else 1900 (fallback)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


BF16_PEAK_TFLOPS = _bf16_peak()
MLP_MAX_ROWS = 1 << 19  # network workspace: the whole warm-start batch (266,240 knot rows) in one chunk


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sspcg", choices=["sspcg", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target duration of each CPU baseline timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--problems", type=int, default=0,
                    help="first N problems of the workload only (small profiler captures); 0: all")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm start (and its MPC arm)")
    ap.add_argument("--no-poly", action="store_true", help="skip the polynomial-preconditioner comparison")
    ap.add_argument("--no-full", action="store_true", help="skip the full-cost-block comparison")
    ap.add_argument("--no-paper-stats", action="store_true",
                    help="skip the Fig. 1-3 statistics (spectra and iterations per preconditioner)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer timing")
    ap.add_argument("--train-problems", type=int, default=4096, help="training problems of the warm-start network")
    ap.add_argument("--train-epochs", type=int, default=1)
    ap.add_argument("--train-gammas", type=int, default=49,
                    help="right-hand sides per training problem (its own gamma and seeded N(0, 1) draws)")
    ap.add_argument("--no-mpc", action="store_true", help="skip the MPC workload (16384 problems, 10 re-solves)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small-problem batch (one problem per CTA against one problem per warp)")
    ap.add_argument("--mpc-resolves", type=int, default=10)
    ap.add_argument("--mpc-problems", type=int, default=0, help="first N problems of the MPC batch; 0: all")
    ap.add_argument("--profile", choices=["step", "pcg", "build", "mpc"], default=None,
                    help="for ncu: set up the tuned plan, then run one step (or one PCG launch set, one build, or "
                         "one PCG launch set of the MPC batch, --mpc-problems of it) inside an NVTX range of that "
                         "name, and exit")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_start(rank: int, per_rank: int) -> int:
    """First problem index of a rank: every rank solves its own ``per_rank`` problems (weak scaling,
    no data-path collective)."""
    return rank * per_rank


def max_over_ranks(value: float, world: int) -> float:
    """The largest of the ranks' values (timings): the whole job's time is its slowest rank's."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job solves/s: all ranks' problems over the slowest rank's time."""
    return world * per_rank * steps / (max_ms / 1e3)


def workload_config(w, nprob):
    return {"workload": w.name, "problems_per_gpu": nprob, "N_range": list(w.N_range), "nx_set": list(w.nx_set),
            "nu_rule": "ceil(nx/2)", "h": w.h, "tol": w.tol, "precond": "symmetric stair",
            "start": "lambda0 = 0", "l2": "inputs larger than L2 (working set ~1.4 GB per step, L2 129 MB)"}


def algorithmic_bytes_per_iteration(p) -> int:
    """Bytes one PCG iteration must read (QP-form operator + preconditioner once, plus vectors):
    A (N nx^2), B (N nx nu), diag Q, R ((N+1) nx + N nu), PD ((N+1) nx^2), PE (N nx^2), FP32;
    vectors: 10 passes over (N+1) nx FP32 values."""
    n, N, m, u = p.N + 1, p.N, p.nx, p.nu
    floats = N * m * m + N * m * u + n * m + N * u + n * m * m + N * m * m + 10 * n * m
    return 4 * floats


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"sspcg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def cpu_baseline(probs, target_s: float, tol: float, samples=None):
    """The FP64 oracle (Schur build, preconditioner and PCG per problem, OpenMP over problems) on the host
    cores, built with gcc -O3: a sample of the first problems of the workload, sized so that one pass on all
    cores takes about target_s / 10, timed five times on all cores and five times on one core (a sample a
    core count smaller), median of each.  The oracle also solves ``samples`` (name -> list of problems); their
    solutions, returned beside the timing, give the lambda error of the GPU results on the same problems."""
    from oracle import block
    block.build()
    cores = os.cpu_count() or 1
    run = lambda sub, nt: block.solve_batch(sub, PRECOND, tol, nthreads=nt)
    m = min(64, len(probs))
    while True:
        _, _, _, _, used, dt = run(probs[:m], cores)
        if dt >= target_s / 10 or m >= len(probs):
            break
        m = min(len(probs), max(m + 1, int(m * min(8.0, 1.2 * (target_s / 10) / max(dt, 1e-3)))))
    t_all = statistics.median(run(probs[:m], cores)[5] for _ in range(5))
    m1 = max(4, m // max(1, used))
    t_one = statistics.median(run(probs[:m1], 1)[5] for _ in range(5))
    refs = {}
    for name, sub in (samples or {}).items():
        refs[name] = run(sub, cores)[0]
    base = {"value": m / t_all, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"first {m} of the {len(probs)} problems per pass, median of 5 passes on {used} cores "
                      f"(FP64 Schur build, preconditioner and PCG; gcc -O3)",
            "seconds_per_pass": t_all,
            "one_core": {"value": m1 / t_one, "unit": UNIT, "cores": 1,
                         "sample": f"first {m1} problems per pass, median of 5 passes", "seconds_per_pass": t_one}}
    return base, refs


def lambda_error(got, ref) -> float:
    """Largest relative 2-norm error of GPU solutions against the oracle's over a sample."""
    worst = 0.0
    for g, r in zip(got, ref):
        r = np.asarray(r, dtype=np.float64).ravel()
        nr = np.linalg.norm(r)
        worst = max(worst, float(np.linalg.norm(np.asarray(g, dtype=np.float64).ravel() - r) / (nr if nr else 1.0)))
    return worst


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, each step one pass over the workload (about a second
    on 16 cores for the 4096-problem batch; SSPCG_REF_SAMPLE bounds it to the first problems)."""
    if rank != 0:
        return
    from oracle import block
    block.build()
    w = WORKLOAD
    per_step = min(w.nprob, int(os.environ.get("SSPCG_REF_SAMPLE", str(w.nprob))))
    probs = P.make_workload(w, count=per_step)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        block.solve_batch(probs[:16], PRECOND, w.tol, nthreads=cores)
    times, used = [], 1
    for _ in range(args.steps):
        _, _, _, status, used, dt = block.solve_batch(probs, PRECOND, w.tol, nthreads=cores)
        times.append(dt)
    t = sum(times)
    value = per_step * args.steps / t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(used), "kind": "oracle",
                             "sample": f"first {per_step} of the {w.nprob} problems of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def train_warm_start(args, torch, sspcg, rank):
    """Train the warm-start network (untimed) on plain solves of the manipulator-like and ragged-batch
    generators: ``--train-problems`` problems, each solved for its own gamma and for ``--train-gammas`` - 1
    more seeded N(0, 1) right-hand sides (4096 x 49 = 200,704 solves by default); returns the network, its
    loss history and the number of solves."""
    half = max(1, args.train_problems // 2)
    base = (1 << 20) + rank * args.train_problems  # disjoint from every rank's benchmark problems
    train = [P.make_problem(P.config_key(2, base + i), 64, 14, 7, 0.01) for i in range(half)]
    train += P.make_workload(P.RAGGED_BATCH_4096, count=half, start=base)
    plan = sspcg.sspcg_plan_create([p.N for p in train], [p.nx for p in train], [p.nu for p in train],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, train)
    b.pipeline(PRECOND)
    d = b.dev
    net = sspcg.sspcg_mlp_create(MLP_MAX_ROWS)
    sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(P.mlp_initial_params(0)).cuda())
    # right-hand sides: the problems' own gamma, then seeded N(0, 1) draws; lambda* of each by the batched PCG
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1 << 40)
    gammas, lams = [d["gamma"]], [b.lam.clone()]
    it = torch.zeros_like(b.iters); rr = torch.zeros_like(b.relres); st = torch.zeros_like(b.status)
    for _ in range(1, max(1, args.train_gammas)):
        g = torch.randn(d["gamma"].shape, generator=gen, device="cuda", dtype=torch.float32)
        lam = torch.zeros_like(g)
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, g, lam, it, rr, st)
        gammas.append(g)
        lams.append(lam)
    torch.cuda.synchronize()
    chunk = 32
    starts = list(range(0, plan.nprob, chunk))
    pairs = [(r, s0) for r in range(len(gammas)) for s0 in starts]
    rng = np.random.default_rng(0)
    loss = torch.zeros(len(pairs), dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(args.train_epochs):
        for j in rng.permutation(len(pairs)):
            r, s0 = pairs[j]
            sspcg.sspcg_mlp_train_step(net, plan, int(s0), min(int(s0) + chunk, plan.nprob), d["A"], d["B"], d["qd"],
                                       d["rd"], gammas[r], b.D, b.E, b.PD, lams[r], sspcg.adam(), loss[j:j + 1])
        hist.append(float(loss.mean().item()))
    return net, hist, len(train) * len(gammas)


def timed_steps(torch, stream, fn, steps, warmup):
    """Mean ms of ``steps`` calls of fn on ``stream`` after ``warmup`` untimed ones (CUDA events)."""
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def warm_start_comparison(args, torch, sspcg, stream, rank, net, sample=64):
    """Held-out warm-start workload (4096 problems, nx = 14, N = 64, h = 0.01): the whole path from lambda0 = 0
    against the whole path started from the trained network (inference inside the timed step), same GPU.
    Returns the results and the sampled problems with each arm's lambda."""
    w = P.WARMSTART_EVAL_4096
    probs = P.make_workload(w, count=w.nprob, start=rank_start(rank, w.nprob))
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=w.tol))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_plan_autotune(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD, b.PE,
                              b.lam, b.iters, b.relres, b.status, stream, which="pipeline")

    def plain():
        sspcg.sspcg_pipeline_batched(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD,
                                     b.PE, b.lam, b.iters, b.relres, b.status, stream)

    def warm():
        sspcg.sspcg_pipeline_warm_batched(plan, net, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E,
                                          b.PD, b.PE, b.lam, b.iters, b.relres, b.status, stream)

    out, lams = {}, {}
    for name, fn in (("plain", plain), ("warm", warm)):
        ms = timed_steps(torch, stream, fn, args.steps, max(3, args.warmup))
        it = b.iters.cpu().numpy()
        ok = bool((b.status.cpu().numpy() == 0).all() and (b.relres.cpu().numpy() <= w.tol).all())
        out[name] = {"solves_per_s": len(probs) / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(it.mean()),
                     "iters_p50": float(np.percentile(it, 50)), "all_converged": ok}
        lams[name] = b.lambdas()[:sample]
    # inference alone (features + three products + scatter), each product engine
    b.pipeline(PRECOND, stream)
    lam0 = plan.empty(sspcg.ARRAY_VEC)
    rows = sum(p.n for p in probs)
    infer = {}
    for engine in ("tcgen05", "mma_sync"):
        sspcg.sspcg_mlp_set_engine(net, engine)
        ms = timed_steps(torch, stream, lambda: sspcg.sspcg_mlp_infer(net, plan, d["A"], d["B"], d["qd"], d["rd"],
                                                                       d["gamma"], b.PD, lam0, stream),
                         args.steps, 3)
        infer[engine] = {"ms": ms, "tflops": rows * MLP_FLOP_PER_ROW / (ms / 1e3) / 1e12,
                         "frac_of_bf16_peak": rows * MLP_FLOP_PER_ROW / (ms / 1e3) / 1e12 / BF16_PEAK_TFLOPS}
    sspcg.sspcg_mlp_set_engine(net, "tcgen05")
    stats = sspcg.plan_stats(plan)
    chunks = -(-rows // MLP_MAX_ROWS)
    return ({"workload": w.name, "plain": out["plain"], "warm": out["warm"],
             "inference": {"rows": rows, "flop_per_row": MLP_FLOP_PER_ROW, "peak_tflops": BF16_PEAK_TFLOPS, **infer},
             "speedup": out["warm"]["solves_per_s"] / out["plain"]["solves_per_s"],
             "gpu_launches": args.steps * (2 * step_launches(probs, stats) + 5 * chunks)},
            probs[:sample], lams)


def step_launches(probs, stats):
    """Kernel launches of one pipeline step: every problem's Schur blocks in one launch, the D_k^-1 blocks in
    one launch per nx, the off-diagonal preconditioner blocks in one launch; the FP64 subset (at most 192
    unknowns) adds its Schur launch, one D_k^-1 launch per nx and its off-diagonal launch; then one PCG
    launch per group."""
    nxs = {p.nx for p in probs}
    tiny_nx = {p.nx for p in probs if (p.N + 1) * p.nx <= 192}
    fp64 = 2 + len(tiny_nx) if stats["pipeline_f64"] else 0
    return 2 + len(nxs) + fp64 + stats["pipeline_launches"]


def poly_comparison(args, torch, sspcg, stream, probs, w):
    """Polynomial preconditioners (Eq. polynomial_precon) on the benchmark workload: the whole pipeline step
    with Phi_d^-1 = sum_{j<=d} (I - Phi^-1 S)^j Phi^-1 for the symmetric stair at d = 0..3, and block-Jacobi
    at d = 1 (the same preconditioner as the symmetric stair at d = 0, applied implicitly from D^-1 and S);
    and the symmetric stair with single-reduction (Chronopoulos-Gear) PCG."""
    out = {}
    # (kind, degree, single-reduction PCG): the last entry is the textbook-equivalent single-reduction variant
    for kind, deg, cg in (("sym", 0, 0), ("sym", 1, 0), ("sym", 2, 0), ("sym", 3, 0), ("bj", 1, 0), ("sym", 0, 1)):
        plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                       sspcg.options(tol=w.tol, poly_degree=deg, cg_variant=cg))
        b = sspcg.Batch(plan, probs)
        d = b.dev

        def step():
            sspcg.sspcg_pipeline_batched(plan, kind, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD,
                                         b.PE, b.lam, b.iters, b.relres, b.status, stream)

        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        it = b.iters.cpu().numpy()
        out[f"{kind}_d{deg}" + ("_single_reduction_cg" if cg else "")] = {
            "solves_per_s": len(probs) / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(it.mean()),
            "all_converged": bool((b.status.cpu().numpy() == 0).all())}
        del b, plan
    return out


def paper_statistics(torch, sspcg, seeds=(16, 3)):
    """The statistics of the paper's Fig. 1 (eigenvalues of Phi_add^-1 S and Phi_sym^-1 S), Fig. 2 (condition
    number of Phi^-1 S relative to Jacobi) and Fig. 3 (PCG iterations relative to Jacobi) on the synthetic
    pendulum-like (nx = 2, N = 20, tol 1e-8) and manipulator-like (nx = 14, N = 64, h = 0.01, tol 1e-6)
    single-solve workloads.  Blocks and iterations come from the GPU (single-problem C-ABI calls, FP64 for
    problems of at most 192 unknowns as in the batched pipeline, FP32 otherwise); spectra from those blocks in
    FP64 on the host, as eig(L^T S L) with Phi^-1 = L L^T."""
    kinds = ("jacobi", "bj", "add", "sym")

    def dense_bt(p, Dd, Eo):
        n, m = p.n, p.nx
        d = Dd.cpu().numpy()[:n * m * m].reshape(n, m, m).astype(np.float64)
        M = np.zeros((n * m, n * m))
        for k in range(n):
            M[k * m:(k + 1) * m, k * m:(k + 1) * m] = d[k]
        if p.N:
            e = Eo.cpu().numpy()[:p.N * m * m].reshape(p.N, m, m).astype(np.float64)
            for k in range(1, n):
                M[k * m:(k + 1) * m, (k - 1) * m:k * m] = e[k - 1]
                M[(k - 1) * m:k * m, k * m:(k + 1) * m] = e[k - 1].T
        return M

    out = {}
    for w, count in ((P.PENDULUM_SINGLE, seeds[0]), (P.MANIPULATOR_SINGLE, seeds[1])):
        rows = {k: {"kappa": [], "iters": [], "ev_min": [], "ev_max": [], "at_one": []} for k in kinds}
        for p in P.make_workload(w, count=count):
            n, m = p.n, p.nx
            f64 = n * m <= 192
            rt = torch.float64 if f64 else torch.float32
            dv = lambda a: torch.from_numpy(np.ascontiguousarray(a) if a.size else np.zeros(4, np.float32)).cuda()
            A, B, qd, rd, g = dv(p.A), dv(p.B), dv(p.qd), dv(p.rd), dv(p.gamma)
            D = torch.zeros(max(n * m * m, 4), dtype=rt, device="cuda")
            E = torch.zeros(max(p.N * m * m, 4), dtype=rt, device="cuda")
            (sspcg.sspcg_build_schur_f64 if f64 else sspcg.sspcg_build_schur)(p.N, m, p.nu, A, B, qd, rd, D, E)
            S = dense_bt(p, D, E)
            for kind in kinds:
                PD, PE = torch.zeros_like(D), torch.zeros_like(E)
                st = torch.zeros(1, dtype=torch.int32, device="cuda")
                (sspcg.sspcg_build_precond_f64 if f64 else sspcg.sspcg_build_precond)(p.N, m, kind, D, E, PD, PE, st)
                lam = torch.zeros(max(n * m, 4), dtype=rt, device="cuda")
                it = torch.zeros(1, dtype=torch.int32, device="cuda")
                rr = torch.zeros(1, dtype=torch.float64, device="cuda")
                (sspcg.sspcg_solve_qp_f64 if f64 else sspcg.sspcg_solve_qp)(
                    p.N, m, p.nu, A, B, qd, rd, PD, PE, g, lam, sspcg.options(tol=w.tol), it, rr, st)
                torch.cuda.synchronize()
                if int(st.item()) != 0:
                    raise RuntimeError(f"paper statistics: solve status {int(st.item())} ({w.name}, {kind})")
                L = np.linalg.cholesky(dense_bt(p, PD, PE))
                ev = np.linalg.eigvalsh(L.T @ S @ L)
                r = rows[kind]
                r["kappa"].append(ev[-1] / ev[0]); r["iters"].append(int(it.item()))
                r["ev_min"].append(ev[0]); r["ev_max"].append(ev[-1])
                r["at_one"].append(float(np.mean(np.abs(ev - 1) <= 1e-5)))
        kj, ij = np.array(rows["jacobi"]["kappa"]), np.array(rows["jacobi"]["iters"], dtype=float)
        res = {"problems": count, "tol": w.tol}
        for kind in kinds:
            r = rows[kind]
            res[kind] = {"kappa_median": float(np.median(r["kappa"])),
                         "kappa_rel_jacobi_median": float(np.median(np.array(r["kappa"]) / kj)),
                         "iters_mean": float(np.mean(r["iters"])),
                         "iters_rel_jacobi_median": float(np.median(np.array(r["iters"]) / ij)),
                         "eig_range": [float(min(r["ev_min"])), float(max(r["ev_max"]))],
                         "eigs_at_one_fraction": float(np.mean(r["at_one"]))}
        ks, ka = np.array(rows["sym"]["kappa"]), np.array(rows["add"]["kappa"])
        its, ita = np.array(rows["sym"]["iters"], dtype=float), np.array(rows["add"]["iters"], dtype=float)
        res["sym_vs_add"] = {"kappa_reduction_median": float(np.median(1 - ks / ka)),
                             "iters_reduction_median": float(np.median(1 - its / ita))}
        out[w.name] = res
    out["paper_context"] = ("Sec. V on its pendulum, cart-pole and manipulator problems: condition number 76-89 % "
                            "below Jacobi and 33-34 % below the additive stair; PCG iterations 51-68 % below "
                            "Jacobi and 17-25 % below the additive stair")
    return out


def full_cost_comparison(args, torch, sspcg, stream, probs, w):
    """Full SPD cost blocks (Q_k = diag(qd_k) + M M^T / nx, R_k likewise) on the benchmark workload: the whole
    step (full-cost Schur build, symmetric stair, block-form PCG) against the same block-form step on the
    diagonal-cost blocks."""
    QR = [P.full_cost(p) for p in probs]
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=w.tol))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    Q = torch.from_numpy(plan.pack(sspcg.ARRAY_DIAG, [q for q, _ in QR])).cuda()
    R = torch.from_numpy(plan.pack(sspcg.ARRAY_RFULL, [r for _, r in QR])).cuda()
    st_b = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")

    def solve():
        sspcg.sspcg_build_precond_batched(plan, PRECOND, b.D, b.E, b.PD, b.PE, st_b, stream)
        sspcg.sspcg_solve_batched(plan, b.D, b.E, b.PD, b.PE, d["gamma"], b.lam, b.iters, b.relres, b.status, stream)

    def full_step():
        sspcg.sspcg_build_schur_full_batched(plan, d["A"], d["B"], Q, R, b.D, b.E, st_b, stream)
        solve()

    def diag_step():
        sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E, stream)
        solve()

    out = {}
    for name, fn in (("full_cost", full_step), ("diagonal_cost", diag_step)):
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        it = b.iters.cpu().numpy()
        out[name] = {"solves_per_s": len(probs) / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(it.mean()),
                     "all_converged": bool((b.status.cpu().numpy() == 0).all() and (st_b.cpu().numpy() == 0).all())}
    out["operator"] = "block form (D, E); the factored QP form needs diagonal Q and R"
    return out


def mpc_comparison(args, torch, sspcg, stream, rank, net=None, sample=32):
    """MPC workload: 16384 problems (N ~ U{64..512}, nx ~ U{4..28}) whose gamma is perturbed by 1 % for each of
    ``--mpc-resolves`` sequential re-solves.  Blocks and preconditioner are built once (A, B, Q, R do not
    change); each re-solve is one PCG launch set (autotuned) from lambda0 = 0 (plain), from the previous
    solution (previous), or from the learned network's lambda0 = MLP(features with the new gamma), inference
    inside the timed re-solve (mlp); warm starts use the fallback to zero.  Most of these problems do not fit
    in shared memory: their blocks stream from L2/HBM, so the roofline is the measured HBM copy bandwidth.
    Returns the results and, per arm, the final re-solve's lambda of ``sample`` spread problems."""
    import dataclasses
    w = P.MPC_BATCH_16384
    t0 = time.time()
    count = args.mpc_problems if args.mpc_problems > 0 else w.nprob
    probs = P.make_workload_parallel(w, count=count, start=rank_start(rank, count))
    gen_s = time.time() - t0
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=w.tol, warm_start=2))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    R = args.mpc_resolves
    # gamma of re-solve 0 warms up (and starts the previous-solution chain); re-solves 1..R are timed
    gammas = [torch.from_numpy(plan.pack(sspcg.ARRAY_VEC, [P.perturb_gamma(p, r) for p in probs])).cuda()
              for r in range(R + 1)]
    t0 = time.time()
    sspcg.sspcg_plan_autotune(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], gammas[0], b.D, b.E, b.PD, b.PE,
                              b.lam, b.iters, b.relres, b.status, stream, which="solve")
    tune_s = time.time() - t0
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E, stream)
        sspcg.sspcg_build_precond_batched(plan, PRECOND, b.D, b.E, b.PD, b.PE, b.status, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    idx = np.linspace(0, len(probs) - 1, sample).astype(int)

    def solve(g):
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, g, b.lam, b.iters, b.relres,
                                     b.status, stream)

    def infer(g):
        sspcg.sspcg_mlp_infer(net, plan, d["A"], d["B"], d["qd"], d["rd"], g, b.PD, b.lam, stream)

    out, lams = {}, {}
    for mode in ("plain", "previous", "mlp"):
        if mode == "mlp" and net is None:
            continue
        b.lam.zero_()
        with torch.cuda.stream(stream):
            solve(gammas[0])  # warm-up (also the start of the previous-solution chain)
        torch.cuda.synchronize()
        iters, ok, alg = [], True, 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for r in range(1, R + 1):
            if mode == "plain":
                b.lam.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            if mode == "mlp":
                infer(gammas[r])
            solve(gammas[r])
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            it = b.iters.cpu().numpy().astype(np.int64)
            ok &= bool((b.status.cpu().numpy() == 0).all() and (b.relres.cpu().numpy() <= w.tol).all())
            iters.append(float(it.mean()))
            alg += sum(int(it[i]) * algorithmic_bytes_per_iteration(p) for i, p in enumerate(probs))
        gbs = alg / (ms / 1e3) / 1e9
        out[mode] = {"solves_per_s": len(probs) * R / (ms / 1e3), "ms_per_resolve": ms / R,
                     "iters_mean_per_resolve": [round(x, 2) for x in iters], "all_converged": ok,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                  "frac": gbs / HBM_PEAK_GBS, "peak_source": HBM_PEAK_SOURCE,
                                  "note": "algorithmic bytes over the re-solve time: every block read counted as "
                                          "if it came from HBM (an upper bound on the HBM rate)"}}
        allx = b.lambdas()
        lams[mode] = [allx[i] for i in idx]
    out["single_reduction"] = implicit_comparison(args, torch, sspcg, stream, probs, b, gammas)
    stats = sspcg.plan_stats(plan)
    last = [dataclasses.replace(probs[i], gamma=P.perturb_gamma(probs[i], R)) for i in idx]
    res = {"workload": w.name, "problems": len(probs), "resolves": R, "generate_seconds": round(gen_s, 1),
           "tune_seconds": round(tune_s, 2), "build_ms": build_ms, **out,
           "speedup_previous": out["previous"]["solves_per_s"] / out["plain"]["solves_per_s"],
           "streamed_problems": stats["solve_qp_stream"], "pcg_launches_per_resolve": stats["solve_qp_launches"]}
    if "mlp" in out:
        res["speedup_mlp"] = out["mlp"]["solves_per_s"] / out["plain"]["solves_per_s"]
    return res, last, lams


def one_time_bytes(probs) -> int:
    """Bytes one PCG launch set must move at least once: read A, B, diag Q, R, PD, PE and gamma, write lambda
    (FP32).  DRAM traffic near this figure means every block was read from HBM once per solve."""
    tot = 0
    for p in probs:
        n, N, m, u = p.N + 1, p.N, p.nx, p.nu
        tot += N * m * m + N * m * u + n * m + N * u + n * m * m + N * m * m + 2 * n * m
    return 4 * tot


def profile_mpc(args, torch, sspcg, stream):
    """One PCG launch set of the MPC batch (its first ``--mpc-problems`` problems, from lambda0 = 0, autotuned)
    inside the NVTX range "mpc", after one untimed launch set."""
    w = P.MPC_BATCH_16384
    count = args.mpc_problems if args.mpc_problems > 0 else w.nprob
    probs = P.make_workload_parallel(w, count=count, start=0)
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=w.tol))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_plan_autotune(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD, b.PE,
                              b.lam, b.iters, b.relres, b.status, stream, which="solve")
    with torch.cuda.stream(stream):
        sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E, stream)
        sspcg.sspcg_build_precond_batched(plan, PRECOND, b.D, b.E, b.PD, b.PE, b.status, stream)

    def solve():
        b.lam.zero_()
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, d["gamma"], b.lam, b.iters,
                                     b.relres, b.status, stream)

    with torch.cuda.stream(stream):
        solve()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("mpc")
    with torch.cuda.stream(stream):
        solve()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    its = b.iters.cpu().numpy().astype(np.int64)
    alg = sum(int(its[i]) * algorithmic_bytes_per_iteration(p) for i, p in enumerate(probs))
    stats = sspcg.plan_stats(plan)
    print(json.dumps({"profile": "mpc", "problems": len(probs), "iters_sum": int(its.sum()),
                      "pcg_algorithmic_bytes": alg, "one_time_bytes": one_time_bytes(probs),
                      "pcg_launches": stats["solve_qp_launches"], "streamed_problems": stats["solve_qp_stream"],
                      "all_converged": bool((b.status.cpu().numpy() == 0).all())}), flush=True)


def small_problems_comparison(args, torch, sspcg, stream, steps=5):
    """The small-problem batch (16384 problems, N ~ U{8..32}, nx in {2, 4, 6}: more problems than the GPU holds
    at one problem per CTA), whole pipeline step: the untuned schedule (one problem per CTA), the autotuned one
    (whose candidates include one problem per warp) and the "warp" schedule (one problem per warp, as many
    warps per CTA as fit), each with its own plan, timed like the headline step."""
    w = P.SMALL_BATCH_16384
    probs = P.make_workload_parallel(w)
    out = {"workload": w.name, "problems": len(probs)}
    for name, sched, tune in (("cta", "auto", False), ("tuned", "auto", True), ("warp", "warp", False)):
        if tune:
            sspcg.sspcg_autotune_cache_clear()
        plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                       sspcg.options(tol=w.tol, schedule=sched))
        b = sspcg.Batch(plan, probs)
        d = b.dev
        if tune:
            sspcg.sspcg_plan_autotune(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD,
                                      b.PE, b.lam, b.iters, b.relres, b.status, stream, which="pipeline")
        ms = timed_steps(torch, stream, lambda: b.pipeline(PRECOND, stream), steps, 3)
        sched_rows = sspcg.sspcg_plan_schedule(plan) + sspcg.sspcg_plan_schedule(plan, "pipeline_f64")
        out[name] = {"solves_per_s": len(probs) / (ms / 1e3), "ms_per_step": ms,
                     "iters_mean": float(b.iters.cpu().numpy().mean()),
                     "all_converged": bool((b.status.cpu().numpy() == 0).all()),
                     "groups_one_problem_per_warp": sum(1 for g in sched_rows if g["warps"] > 0),
                     "groups": len(sched_rows)}
        del b, plan
    sspcg.sspcg_autotune_cache_clear()
    out["warp_vs_cta"] = out["warp"]["solves_per_s"] / out["cta"]["solves_per_s"]
    return out


def build_bytes(probs) -> int:
    """HBM bytes the two build calls must move at least: read A, B, diag Q, diag R once, write the Schur blocks
    D, E and the preconditioner blocks PD, PE once (FP32)."""
    tot = 0
    for p in probs:
        n, N, m, u = p.N + 1, p.N, p.nx, p.nu
        tot += N * m * m + N * m * u + n * m + N * u + 2 * (n * m * m + N * m * m)
    return 4 * tot


def implicit_comparison(args, torch, sspcg, stream, probs, b, gammas, resolves=3):
    """Single-reduction (Chronopoulos-Gear) PCG on the MPC workload, with the symmetric stair applied explicitly
    (PD and PE blocks) or implicitly, Phi_sym^-1 = 2 D^-1 - D^-1 S D^-1: block-Jacobi D^-1 with the degree-1
    polynomial and no PE blocks.  Re-solves from lambda0 = 0 on the blocks the MPC section built (its PD is
    D^-1 for both), each plan autotuned for its own launch shapes."""
    d = b.dev
    out = {}
    for name, kind, deg, pe in (("explicit", "sym", 0, b.PE), ("implicit", "bj", 1, None)):
        plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                       sspcg.options(tol=P.MPC_BATCH_16384.tol, cg_variant=1, poly_degree=deg))
        lam = torch.zeros_like(b.lam); it = torch.zeros_like(b.iters); rr = torch.zeros_like(b.relres)
        st = torch.zeros_like(b.status)
        D2, E2 = torch.zeros_like(b.D), torch.zeros_like(b.E)
        PD2, PE2 = torch.zeros_like(b.PD), torch.zeros_like(b.PE)
        sspcg.sspcg_plan_autotune(plan, kind, d["A"], d["B"], d["qd"], d["rd"], gammas[0], D2, E2, PD2, PE2, lam, it,
                                  rr, st, stream, which="solve")
        del D2, E2, PD2, PE2
        ms, iters, ok = 0.0, [], True
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for r in range(1, resolves + 1):
            lam.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, pe, gammas[r], lam, it, rr, st,
                                         stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            iters.append(float(it.cpu().numpy().mean()))
            ok &= bool((st.cpu().numpy() == 0).all())
        out[name] = {"solves_per_s": len(probs) * resolves / (ms / 1e3), "ms_per_resolve": ms / resolves,
                     "iters_mean": round(float(np.mean(iters)), 2), "all_converged": ok}
        del plan
    out["implicit_vs_explicit"] = out["implicit"]["solves_per_s"] / out["explicit"]["solves_per_s"]
    return out


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2309_06427_gb300 import build as _build
    _build.build()
    from paper_2309_06427_gb300 import sspcg

    if args.profile == "mpc":
        profile_mpc(args, torch, sspcg, torch.cuda.Stream())
        return

    w = WORKLOAD
    nprob = args.problems if args.problems > 0 else w.nprob
    probs = P.make_workload(w, count=nprob, start=rank_start(rank, nprob))  # weak scaling
    opts = sspcg.options(tol=w.tol)
    stream = torch.cuda.Stream()
    warm = max(3, args.warmup)
    smem_4 = sspcg.sspcg_measure_smem_bandwidth(4, 8192)
    smem_16 = sspcg.sspcg_measure_smem_bandwidth(16, 8192)
    smem_peak = max(smem_4, smem_16)

    # the schedule the library picks without tuning (timed for comparison), then the autotuned plan whose
    # pipeline, captured in one CUDA graph, is the timed step
    plan_h = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs], opts)
    bh = sspcg.Batch(plan_h, probs)
    heuristic_ms = timed_steps(torch, stream, lambda: bh.pipeline(PRECOND, stream), args.steps, warm)
    del bh, plan_h
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs], opts)
    b = sspcg.Batch(plan, probs, pin=True)
    d = b.dev
    t0 = time.time()
    sspcg.sspcg_plan_autotune(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD, b.PE,
                              b.lam, b.iters, b.relres, b.status, stream)
    tune_s = time.time() - t0
    b.capture(PRECOND, stream)

    def step():
        sspcg.sspcg_plan_launch(plan, stream)

    if args.profile:
        # one profiled region (ncu --nvtx --nvtx-include "<name>/"), after one untimed step
        it_p = torch.zeros_like(b.iters); rr_p = torch.zeros_like(b.relres); st_p = torch.zeros_like(b.status)
        lam_p = torch.zeros_like(b.lam)
        fn = {"step": step,
              "pcg": lambda: sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE,
                                                          d["gamma"], lam_p, it_p, rr_p, st_p, stream),
              "build": lambda: (sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E,
                                                                stream),
                                sspcg.sspcg_build_precond_batched(plan, PRECOND, b.D, b.E, b.PD, b.PE, st_p, stream))}
        with torch.cuda.stream(stream):
            if args.profile == "pcg":  # FP32 blocks for every problem (the pipeline builds the smallest in FP64)
                fn["build"]()
            fn[args.profile]()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(args.profile)
        with torch.cuda.stream(stream):
            fn[args.profile]()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        its = (it_p if args.profile == "pcg" else b.iters).cpu().numpy().astype(np.int64)
        alg = sum(int(its[i]) * algorithmic_bytes_per_iteration(p) for i, p in enumerate(probs))
        print(json.dumps({"profile": args.profile, "problems": nprob, "iters_sum": int(its.sum()),
                          "pcg_algorithmic_bytes": alg, "one_time_bytes": one_time_bytes(probs),
                          "build_bytes": build_bytes(probs),
                          "pcg_launches": sspcg.plan_stats(plan)["solve_qp_launches"]}), flush=True)
        return

    with torch.cuda.stream(stream):
        for _ in range(warm):
            step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), world)

    iters = b.iters.cpu().numpy().astype(np.int64)
    status = b.status.cpu().numpy()
    relres = b.relres.cpu().numpy()
    ok = bool((status == 0).all() and (relres <= w.tol).all())
    value = job_throughput(world, nprob, args.steps, total_ms)
    sample3 = list(range(min(256, nprob)))
    lam_main = b.lambdas()
    lam_main = [lam_main[i] for i in sample3]

    # The phases timed apart: the PCG launches alone (FP32, every problem, all groups concurrently) on the
    # blocks the pipeline built, and the two build calls alone.
    it_d = torch.zeros_like(b.iters); rr_d = torch.zeros_like(b.relres); st_d = torch.zeros_like(b.status)
    lam_d = torch.zeros_like(b.lam)

    def pcg_only():
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, d["gamma"], lam_d, it_d,
                                     rr_d, st_d, stream)

    def build_only():
        sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E, stream)
        sspcg.sspcg_build_precond_batched(plan, PRECOND, b.D, b.E, b.PD, b.PE, st_d, stream)

    build_ms = timed_steps(torch, stream, build_only, args.steps, 1)
    pcg_ms = timed_steps(torch, stream, pcg_only, args.steps, 1)
    # roofline of the dominant kernel (the PCG launches): algorithmic bytes per launch set / its time
    iters_pcg = it_d.cpu().numpy().astype(np.int64)
    alg_bytes = sum(int(iters_pcg[i]) * algorithmic_bytes_per_iteration(p) for i, p in enumerate(probs))
    achieved_gbs = alg_bytes / (pcg_ms / 1e3) / 1e9
    bb = build_bytes(probs)
    build_gbs = bb / (build_ms / 1e3) / 1e9

    h2d = d2h = 0
    e2e_ms = e2e_sync_ms = None
    e2e_ok = None
    if not args.no_e2e:
        # end to end through the host-buffer C-ABI call (copies inside the timed region): the asynchronous
        # entry point overlaps one step's host-to-device copy with the previous step's compute; the
        # synchronous one (copy in, compute, copy out, wait) is timed beside it
        h = b.host
        lam_h = torch.zeros(max(int(plan.sizes[sspcg.ARRAY_VEC]), 4)).pin_memory()
        it_h = torch.zeros(plan.nprob, dtype=torch.int32).pin_memory()
        rr_h = torch.zeros(plan.nprob, dtype=torch.float64).pin_memory()
        st_h = torch.zeros(plan.nprob, dtype=torch.int32).pin_memory()
        host_args = (plan, PRECOND, h["A"], h["B"], h["qd"], h["rd"], h["gamma"], lam_h, it_h, rr_h, st_h, stream)

        def e2e_timed(call, join):
            with torch.cuda.stream(stream):
                for _ in range(warm):
                    call(*host_args)
                join()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    call(*host_args)
                join()
                e1.record(stream)
                torch.cuda.synchronize()
            return max_over_ranks(e0.elapsed_time(e1), world)

        e2e_sync_ms = e2e_timed(sspcg.sspcg_pipeline_host, lambda: None)
        e2e_ms = e2e_timed(sspcg.sspcg_pipeline_host_async, lambda: sspcg.sspcg_plan_join(plan, stream))
        e2e_ok = bool((st_h.numpy() == 0).all()) and torch.equal(lam_h, b.lam.cpu())
        h2d = sum(int(h[k].numel()) * 4 for k in ("A", "B", "qd", "rd", "gamma"))
        d2h = int(lam_h.numel()) * 4 + plan.nprob * (4 + 4 + 8)

    if rank != 0:
        if world > 1:
            dist.barrier()
        return
    stats = sspcg.plan_stats(plan)
    sched = sspcg.sspcg_plan_schedule(plan, "pipeline") + sspcg.sspcg_plan_schedule(plan, "pipeline_f64")
    traffic = pcg_traffic() if nprob == w.nprob else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, nprob),
        "iters": {"mean": float(iters.mean()), "min": int(iters.min()), "max": int(iters.max()),
                  "p50": float(np.percentile(iters, 50)), "p90": float(np.percentile(iters, 90))},
        "all_converged": ok,
        "pcg_ms_per_step": pcg_ms,
        "roofline": {"bound": "smem", "achieved": achieved_gbs, "peak": smem_peak, "unit": "GB/s",
                     "frac": achieved_gbs / smem_peak, "traffic": traffic,
                     "traffic_note": "DRAM bytes per PCG launch set of the batch (ncu, profiles/); the blocks are "
                                     "read from shared memory and L2, so HBM traffic is far below the "
                                     "algorithmic bytes",
                     "kernel": "pcg_kernel (all FP32 PCG launches of the batch, timed alone)",
                     "peak_source": "measured: sspcg_measure_smem_bandwidth, conflict-free shared-memory reads "
                                    "on every SM (the better of 32-bit and 128-bit loads)",
                     "peak_measured_lds32_gbs": smem_4, "peak_measured_lds128_gbs": smem_16,
                     "frac_of_derived_peak": achieved_gbs / (torch.cuda.get_device_properties(local)
                                                             .multi_processor_count * SMEM_BYTES_PER_CLK_PER_SM *
                                                             (clk.get("sm_max_mhz") or 2070.0) * 1e-3)},
        "build": {"ms_per_step": build_ms, "roofline": {"bound": "hbm", "achieved": build_gbs, "peak": HBM_PEAK_GBS,
                                                        "unit": "GB/s", "frac": build_gbs / HBM_PEAK_GBS,
                                                        "bytes": bb, "peak_source": HBM_PEAK_SOURCE}},
        "gpu_launches": args.steps * step_launches(probs, stats),
        "clocks": clk,
    }
    if e2e_ms is not None:
        line["e2e"] = {"value": job_throughput(world, nprob, args.steps, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "entry": "sspcg_pipeline_host_async (two device slots, copies overlapped with the previous "
                                "step's compute)", "results_match_device_path": e2e_ok,
                       "synchronous": job_throughput(world, nprob, args.steps, e2e_sync_ms)}
    line["schedules"] = {"autotune_seconds": round(tune_s, 2), "step": "one CUDA graph (sspcg_plan_launch)",
                         "heuristic_ms_per_step": heuristic_ms, "tuned_ms_per_step": total_ms / args.steps,
                         "resident_fp32_problems": stats["pipeline_resident"],
                         "streamed_fp32_problems": stats["pipeline_stream"], "fp64_problems": stats["pipeline_f64"],
                         "pcg_launches_per_step": stats["pipeline_launches"],
                         "groups": [{k: g[k] for k in ("nx", "cls", "problems", "max_N", "block", "grid", "stream",
                                                       "share", "warps")}
                                    for g in sched]}

    # the FP64 reduction mode beside the double-float default
    plan_r = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                     sspcg.options(tol=w.tol, reduction="f64"))
    br = sspcg.Batch(plan_r, probs)
    dr = br.dev
    sspcg.sspcg_plan_autotune(plan_r, PRECOND, dr["A"], dr["B"], dr["qd"], dr["rd"], dr["gamma"], br.D, br.E, br.PD,
                              br.PE, br.lam, br.iters, br.relres, br.status, stream, which="pipeline")
    ms_r = timed_steps(torch, stream, lambda: br.pipeline(PRECOND, stream), args.steps, warm)
    lam_r = br.lambdas()
    line["reduction_f64"] = {"solves_per_s": nprob / (ms_r / 1e3), "ms_per_step": ms_r,
                             "iters_mean": float(br.iters.cpu().numpy().mean()),
                             "all_converged": bool((br.status.cpu().numpy() == 0).all()),
                             "note": "alpha/beta dot products in native FP64 instead of double-float"}
    lam_r = [lam_r[i] for i in sample3]
    del br, plan_r

    if not args.no_poly:
        line["polynomial_preconditioners"] = poly_comparison(args, torch, sspcg, stream, probs, w)
    if not args.no_full:
        line["full_cost_blocks"] = full_cost_comparison(args, torch, sspcg, stream, probs, w)
    if not args.no_paper_stats:
        line["paper_statistics"] = paper_statistics(torch, sspcg)
    net = None
    samples = {"ragged": [probs[i] for i in sample3]}
    gpu_lams = {"value": ("ragged", lam_main), "reduction_f64": ("ragged", lam_r)}
    if not args.no_warm_start:
        t0 = time.time()
        net, hist, ntrain = train_warm_start(args, torch, sspcg, rank)
        torch.cuda.synchronize()
        train_s = time.time() - t0
        ws, ws_probs, ws_lams = warm_start_comparison(args, torch, sspcg, stream, rank, net)
        ws.update({"train_problems": args.train_problems, "train_solves": ntrain, "train_epochs": args.train_epochs,
                   "train_loss": [round(x, 4) for x in hist], "train_seconds": round(train_s, 2)})
        line["warm_start"] = ws
        samples["warmstart_eval"] = ws_probs
        gpu_lams["warm_start.plain"] = ("warmstart_eval", ws_lams["plain"])
        gpu_lams["warm_start.warm"] = ("warmstart_eval", ws_lams["warm"])

        # warm start vs plain on the benchmark workload itself (direct launches of both pipelines)
        def plain3():
            sspcg.sspcg_pipeline_batched(plan, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD,
                                         b.PE, b.lam, b.iters, b.relres, b.status, stream)

        def warm3():
            sspcg.sspcg_pipeline_warm_batched(plan, net, PRECOND, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D,
                                              b.E, b.PD, b.PE, b.lam, b.iters, b.relres, b.status, stream)

        r3 = {}
        for name, fn in (("plain", plain3), ("warm", warm3)):
            ms = timed_steps(torch, stream, fn, args.steps, warm)
            r3[name] = {"solves_per_s": nprob / (ms / 1e3), "ms_per_step": ms,
                        "iters_mean": float(b.iters.cpu().numpy().mean()),
                        "all_converged": bool((b.status.cpu().numpy() == 0).all())}
            lw = b.lambdas()
            gpu_lams[f"warm_start_ragged.{name}"] = ("ragged", [lw[i] for i in sample3])
        r3["speedup"] = r3["warm"]["solves_per_s"] / r3["plain"]["solves_per_s"]
        line["warm_start_ragged"] = r3
    if not args.no_small:
        line["small_problems"] = small_problems_comparison(args, torch, sspcg, stream)
    if not args.no_mpc:
        mpc, mpc_probs, mpc_lams = mpc_comparison(args, torch, sspcg, stream, rank, net)
        line["mpc"] = mpc
        samples["mpc_last_resolve"] = mpc_probs
        for k, v in mpc_lams.items():
            gpu_lams[f"mpc.{k}"] = ("mpc_last_resolve", v)
    if world == 1 and not args.no_cpu_baseline:
        base, refs = cpu_baseline(probs, args.cpu_seconds, w.tol, samples)
        line["cpu_baseline"] = base
        line["lambda_error"] = {
            name: {"max_rel": lambda_error(lams, refs[smp]), "problems": len(lams), "sample": smp}
            for name, (smp, lams) in gpu_lams.items()}
        line["lambda_error"]["note"] = ("max over the sampled problems of ||lambda - lambda_oracle|| / "
                                        "||lambda_oracle||; the oracle solves from zero in FP64 to the same tolerance")
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()


if __name__ == "__main__":
    main()
