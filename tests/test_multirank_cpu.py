"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2): each rank
solves its own problems (weak scaling, no data-path collective), the job's time is
the slowest rank's, and only rank 0 reports; the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_2309_06427_gb300 import problems as P
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per_rank = 5
    start = bench.rank_start(rank, per_rank)
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=per_rank, start=start)
    my_ms = 10.0 + 7.0 * rank  # rank 1 is the slow one
    t = bench.max_over_ranks(my_ms, world)
    thr = bench.job_throughput(world, per_rank, 3, t)
    q.put((rank, start, [p.key for p in probs], t, thr))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_problems_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0, k0, t0, thr0), (r1, s1, k1, t1, thr1) = out
    assert (s0, s1) == (0, 5)
    assert not set(k0) & set(k1)  # disjoint problems
    assert t0 == t1 == 17.0  # max over ranks
    assert thr0 == thr1 == pytest.approx(2 * 5 * 3 / 0.017)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Under a 2-rank launch the oracle arm prints one JSON line from rank 0; rank 1 exits 0 without work."""
    env = dict(os.environ, SSPCG_REF_SAMPLE="8", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    outs = []
    for rank in (0, 1):
        e = dict(env, RANK=str(rank), LOCAL_RANK=str(rank))
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                            "--steps", "1", "--warmup", "1"], env=e, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    import json
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert outs[1] == ""
