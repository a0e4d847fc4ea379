"""Seeded input generators: published SplitMix64 values, determinism, shapes."""
import numpy as np

from paper_2309_06427_gb300 import problems as P


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0: the first three outputs of the reference generator
    # (Steele, Lea, Flood 2014; also Vigna's splitmix64.c).
    z = P.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_slices_agree():
    a = P.splitmix64(12345, 10)
    b = P.splitmix64(12345, 4, start=6)
    assert np.array_equal(a[6:], b)


def test_normals_moments():
    z = P.normals(7, 200001)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_problem_shapes_and_determinism():
    p = P.make_problem(P.config_key(1, 0), 20, 2, 1, 0.05)
    q = P.make_problem(P.config_key(1, 0), 20, 2, 1, 0.05)
    assert p.A.shape == (20, 2, 2) and p.B.shape == (20, 2, 1) and p.qd.shape == (21, 2)
    assert p.rd.shape == (20, 1) and p.gamma.shape == (21, 2)
    for a, b in zip((p.A, p.B, p.qd, p.rd, p.gamma), (q.A, q.B, q.qd, q.rd, q.gamma)):
        assert a.dtype == np.float32 and np.array_equal(a, b)
    assert p.qd.min() >= 0.1 and p.qd.max() <= 10 and p.rd.min() >= 0.1 and p.rd.max() <= 1


def test_ragged_workload_shape_distribution():
    w = P.RAGGED_BATCH_4096
    shapes = [P.problem_shape(w, i) for i in range(600)]
    Ns = np.array([s[1] for s in shapes]); nxs = np.array([s[2] for s in shapes])
    assert Ns.min() >= 16 and Ns.max() <= 128
    assert set(nxs.tolist()) == {4, 12, 14, 21}
    assert all(s[3] == (s[2] + 1) // 2 for s in shapes)


def test_gamma_perturbation_is_one_percent():
    p = P.make_problem(P.config_key(5, 3), 64, 4, 2, 0.05)
    g1 = P.perturb_gamma(p, 0)
    rel = (g1 / p.gamma - 1)
    assert 0.005 < rel.std() < 0.015
    assert not np.array_equal(g1, P.perturb_gamma(p, 1))


def test_parallel_generation_matches_serial():
    from paper_2309_06427_gb300 import problems as P
    a = P.make_workload(P.MPC_BATCH_16384, count=20, start=100)
    b = P.make_workload_parallel(P.MPC_BATCH_16384, count=20, start=100, workers=2, chunk=7)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.key == y.key and x.N == y.N and x.nx == y.nx
        for f in ("A", "B", "qd", "rd", "gamma"):
            assert np.array_equal(getattr(x, f), getattr(y, f))
