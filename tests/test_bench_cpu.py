"""Host helpers of bench.py: the kernel-launch count of a step, the guard that ties the recorded PCG
traffic to the kernel source, the per-iteration algorithmic bytes and the whole-job throughput."""
import os
import shutil

import pytest

import bench
from paper_2309_06427_gb300 import problems as P


def test_step_launches_count():
    """Ragged batch: Schur + one D^-1 launch per nx (4) + off-diagonal, the FP64 subset's Schur + one D^-1
    per tiny nx (1) + off-diagonal, and one launch per PCG group (15): 6 + 3 + 15 = 24."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=400)
    nxs = {p.nx for p in probs}
    tiny_nx = {p.nx for p in probs if (p.N + 1) * p.nx <= 192}
    assert nxs == {4, 12, 14, 21} and tiny_nx == {4}
    assert bench.step_launches(probs, {"pipeline_f64": 1, "pipeline_launches": 15}) == 24
    # no FP64 subset: no FP64 build launches
    assert bench.step_launches(probs, {"pipeline_f64": 0, "pipeline_launches": 15}) == 6 + 15


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The recorded DRAM figure is reported only while the kernel source hashes to the value recorded with it."""
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2309_06427_gb300" / "csrc").mkdir(parents=True)
    for f in ("pcg.cuh", "kernels.h"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2309_06427_gb300", "csrc", f),
                    root / "paper_2309_06427_gb300" / "csrc" / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    with open(root / "profiles" / bench.TRAFFIC_FILE, "w") as f:
        f.write(f"pcg_traffic_bytes_per_launch: 123456\nsource_sha256_16: {bench.kernel_source_hash()}\n")
    assert bench.pcg_traffic() == 123456
    # a comment does not change the kernel; code does
    with open(root / "paper_2309_06427_gb300" / "csrc" / "pcg.cuh", "a") as f:
        f.write("\n// a comment\n")
    assert bench.pcg_traffic() == 123456
    with open(root / "paper_2309_06427_gb300" / "csrc" / "pcg.cuh", "a") as f:
        f.write("\nnamespace sspcg { constexpr int kChanged = 1; }\n")
    assert bench.pcg_traffic() is None


def test_algorithmic_bytes_and_throughput():
    p = P.custom_problems([(3, 2, 1)], config=88)[0]
    # A 3*4, B 3*2, diag Q 4*2, diag R 3, PD 4*4, PE 3*4, vectors 10 * 4*2 floats
    assert bench.algorithmic_bytes_per_iteration(p) == 4 * (12 + 6 + 8 + 3 + 16 + 12 + 80)
    # 2 ranks x 100 problems x 10 steps in 20 ms (slowest rank)
    assert bench.job_throughput(2, 100, 10, 20.0) == pytest.approx(100_000.0)
    assert bench.rank_start(3, 4096) == 3 * 4096
