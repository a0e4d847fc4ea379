"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: Schur and preconditioner blocks within 1e-6 (relative Frobenius norm)
of the oracle's FP64 blocks computed from the same inputs; lambda within
1e-5 (relative 2-norm) of the oracle's lambda and iteration counts within 1.
"""
import numpy as np
import pytest
import torch

from oracle import block, dense
from paper_2309_06427_gb300 import problems as P

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2309_06427_gb300 import build as _build
    _build.build()
    from paper_2309_06427_gb300 import sspcg
    from _gpu_helpers import (ITER_TOL, LAMBDA_RTOL, blocks_to_oracle, dev, gpu_precond, gpu_schur,
                              gpu_solve_auto, gpu_solve_qp, gpu_solve_qp_f64, is_tiny, iters_ok, rel)

SHAPES = [(0, 1, 1), (0, 5, 3), (1, 2, 1), (2, 3, 2), (7, 4, 2), (20, 2, 1), (33, 12, 6), (64, 14, 7),
          (17, 21, 11), (9, 28, 14), (40, 5, 1), (3, 1, 2), (100, 4, 2), (25, 7, 4), (12, 9, 0)]


def _probs(shapes, h=0.05, config=55):
    return P.custom_problems(shapes, h=h, config=config)


@pytest.mark.parametrize("p", _probs(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_schur_blocks(p):
    _, D, E = gpu_schur(p)
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    n, m = p.n, p.nx
    Dg = D.cpu().numpy()[:n * m * m].reshape(n, m, m)
    assert rel(Dg, S.d) <= 1e-6
    assert np.array_equal(Dg, np.transpose(Dg, (0, 2, 1)))  # exactly symmetric
    if p.N:
        Eg = E.cpu().numpy()[:p.N * m * m].reshape(p.N, m, m)
        assert rel(Eg, S.l[1:]) <= 1e-6


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _probs(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_preconditioner_blocks(p, kind):
    """sspcg_build_precond against the oracle's preconditioner of the same (FP32) blocks."""
    _, D, E = gpu_schur(p)
    PD, PE, st = gpu_precond(p, D, E, kind)
    assert st == 0
    So = blocks_to_oracle(p, D, E)
    Mo = block.build_precond(So, kind)
    n, m = p.n, p.nx
    PDg = PD.cpu().numpy()[:n * m * m].reshape(n, m, m)
    assert rel(PDg, Mo.d) <= 1e-6
    assert np.array_equal(PDg, np.transpose(PDg, (0, 2, 1)))
    if p.N:
        PEg = PE.cpu().numpy()[:p.N * m * m].reshape(p.N, m, m)
        assert rel(PEg, Mo.l[1:]) <= 1e-6 * max(1.0, np.abs(Mo.d).max() / max(np.abs(Mo.l).max(), 1e-30))
        assert np.allclose(Mo.u[:-1], np.transpose(Mo.l[1:], (0, 2, 1)), atol=1e-12)


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _probs(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_solve_block_form(p, kind):
    """sspcg_solve on the GPU's FP32 blocks == oracle PCG on the same blocks."""
    _, D, E = gpu_schur(p)
    PD, PE, _ = gpu_precond(p, D, E, kind)
    g = dev(p.gamma)
    lam = torch.zeros_like(g)
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve(p.N, p.nx, D, E, PD, PE, g, lam, sspcg.options(tol=1e-6), it, rr, st)
    So = blocks_to_oracle(p, D, E)
    x, it_o, rr_o, _, st_o = block.pcg(So, block.build_precond(So, kind), p.gamma, 1e-6)
    assert int(st.item()) == 0 and st_o == 0
    assert iters_ok(int(it.item()), it_o, fp32_tiny=is_tiny(p), unknowns=p.n * p.nx, kind=kind)
    assert rel(lam.cpu().numpy()[:p.gamma.size], x) <= LAMBDA_RTOL
    assert float(rr.item()) <= 1e-6


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _probs(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_whole_path_qp_form(p, kind):
    """QP data -> lambda on the GPU == the oracle's FP64 path from the same QP data (FP64 path for
    problems of at most 192 unknowns, FP32 otherwise, as the batched pipeline does)."""
    lam, it, rr, st = gpu_solve_auto(p, kind, 1e-6)
    _, _, x, it_o, rr_o, _, st_o = block.solve_problem(p, kind, 1e-6)
    assert st == 0 and st_o == 0
    assert iters_ok(it, it_o, unknowns=p.n * p.nx, kind=None if is_tiny(p) else kind)
    assert rel(lam, x) <= LAMBDA_RTOL
    assert rr <= 1e-6


@pytest.mark.parametrize("p", _probs([s for s in SHAPES if (s[0] + 1) * s[1] <= 192]),
                         ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_fp32_path_on_tiny_problems(p):
    """FP32 on problems of at most 192 unknowns: lambda at the parity bar, iterations bounded."""
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6)
    _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
    assert st == 0 and rr <= 1e-6
    assert iters_ok(it, it_o, fp32_tiny=True)
    assert rel(lam, x) <= LAMBDA_RTOL


@pytest.mark.parametrize("seed", range(8))
def test_manipulator_workload_parity(seed):
    """nx = 14, nu = 7, N = 64, h = 0.01, tol 1e-6: the ill-conditioned case (kappa(S) ~ 2e4)."""
    p = P.make_problem(P.config_key(2, seed), 64, 14, 7, 0.01)
    for kind in ("sym", "add", "bj"):
        lam, it, rr, st = gpu_solve_qp(p, kind, 1e-6)
        _, _, x, it_o, _, _, st_o = block.solve_problem(p, kind, 1e-6)
        assert st == 0 and abs(it - it_o) <= ITER_TOL, (kind, it, it_o)
        assert rel(lam, x) <= LAMBDA_RTOL, kind


def test_pendulum_workload_parity():
    """nx = 2, nu = 1, N = 20, h = 0.05, tol 1e-8 on the FP64 path: the symmetric stair ends in
    exactly 21 iterations (21 distinct eigenvalues, Thm. 4.1/4.2), as in the oracle."""
    p = P.make_workload(P.PENDULUM_SINGLE)[0]
    for kind in ("sym", "add", "bj", "jacobi"):
        lam, it, rr, st = gpu_solve_qp_f64(p, kind, 1e-8)
        _, _, x, it_o, _, _, st_o = block.solve_problem(p, kind, 1e-8)
        assert st == 0 and abs(it - it_o) <= ITER_TOL, (kind, it, it_o)
        assert rel(lam, x) <= 1e-10
        # FP32 path: same answer, more iterations (no finite termination in FP32)
        lam32, it32, rr32, st32 = gpu_solve_qp(p, kind, 1e-8)
        assert st32 == 0 and rr32 <= 1e-8 and rel(lam32, x) <= LAMBDA_RTOL
        assert iters_ok(it32, it_o, fp32_tiny=True)


@pytest.mark.parametrize("reduction", ["df", "f32", "f64"])
@pytest.mark.parametrize("schedule", ["resident", "stream"])
def test_reduction_modes_and_schedules(reduction, schedule):
    for p in _probs([(64, 14, 7), (30, 21, 11), (5, 3, 2)], h=0.01, config=56):
        lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6, reduction=reduction, schedule=schedule)
        _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
        assert st == 0 and iters_ok(it, it_o, fp32_tiny=is_tiny(p))
        assert rel(lam, x) <= LAMBDA_RTOL


@pytest.mark.parametrize("schedule", ["resident", "stream"])
def test_fp64_path_schedules(schedule):
    for p in _probs([(40, 4, 2), (10, 12, 6), (64, 14, 7)], h=0.01, config=64):
        lam, it, rr, st = gpu_solve_qp_f64(p, "sym", 1e-6, schedule=schedule)
        _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
        assert st == 0 and abs(it - it_o) <= ITER_TOL
        assert rel(lam, x) <= 1e-7  # both FP64; they differ by summation order only


def test_schedules_agree_bitwise():
    p = _probs([(50, 12, 6)], config=57)[0]
    a = gpu_solve_qp(p, "sym", 1e-6, schedule="resident", block_threads=128)
    b = gpu_solve_qp(p, "sym", 1e-6, schedule="stream", block_threads=128)
    assert a[1] == b[1] and np.array_equal(a[0], b[0])


def test_maxiter_iterates_match_oracle():
    """Stopping after 5 iterations: the 5th iterate itself matches the oracle's."""
    p = _probs([(30, 6, 3)], config=58)[0]
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-12, max_iter=5)
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    x, it_o, rr_o, _, st_o = block.pcg(S, block.build_precond(S, "sym"), p.gamma, 1e-12, max_iter=5)
    assert st == 1 and st_o == block.MAXITER and it == 5 and it_o == 5
    assert rel(lam, x) <= 1e-5
    assert abs(rr - rr_o) <= 1e-4 * rr_o


def test_zero_rhs_and_exact_warm_start():
    p = _probs([(12, 4, 2)], config=59)[0]
    p0 = P.Problem(p.N, p.nx, p.nu, p.A, p.B, p.qd, p.rd, np.zeros_like(p.gamma))
    lam, it, rr, st = gpu_solve_qp(p0, "sym", 1e-6, lam0=np.ones_like(p.gamma))
    assert it == 0 and st == 0 and not lam.any()
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    xd = dense.cholesky_solve(S.dense(), p.gamma).reshape(p.gamma.shape)
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-4, lam0=xd.astype(np.float32))
    assert st == 0 and it <= 1


def test_warm_start_with_fallback():
    p = _probs([(20, 5, 3)], config=60)[0]
    bad = np.full_like(p.gamma, 1e3)
    cold = gpu_solve_qp(p, "sym", 1e-6)
    warm = gpu_solve_qp(p, "sym", 1e-6, lam0=bad, warm=2)
    assert warm[3] == 0 and warm[1] == cold[1] and np.array_equal(warm[0], cold[0])
    # a good warm start (the oracle's answer perturbed by 1e-3) needs fewer iterations
    _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
    good = (x * (1 + 1e-3 * np.random.default_rng(0).standard_normal(x.shape))).astype(np.float32)
    w2 = gpu_solve_qp(p, "sym", 1e-6, lam0=good, warm=2)
    assert w2[3] == 0 and w2[1] < cold[1]
    assert rel(w2[0], x) <= LAMBDA_RTOL


def test_not_spd_block_is_reported():
    p = _probs([(6, 3, 2)], config=61)[0]
    qd = p.qd.copy(); qd[3, 0] = -2.0
    p2 = P.Problem(p.N, p.nx, p.nu, p.A, p.B, qd, p.rd, p.gamma)
    _, D, E = gpu_schur(p2)
    _, _, st = gpu_precond(p2, D, E, "sym")
    assert st == 3


def test_true_residual_kernel_matches_oracle():
    p = _probs([(40, 9, 5)], config=62)[0]
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6)
    (A, B, qd, rd), _, _ = gpu_schur(p)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sspcg.sspcg_residual_qp(p.N, p.nx, p.nu, A, B, qd, rd, dev(p.gamma), dev(lam), out)
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    g = p.gamma.astype(np.float64).ravel()
    want = np.linalg.norm(g - Sd @ lam.astype(np.float64).ravel()) / np.linalg.norm(g)
    assert abs(out.item() - want) <= 1e-6 * want + 1e-13


def test_inputless_dynamics_nu0():
    """nu = 0 (no inputs, B empty): S = C G^-1 C^T with state rows only, far worse conditioned
    (kappa(Phi_sym^-1 S) ~ 3e3 at N = 40, nx = 5).  FP64 path: oracle parity.  FP32 path: lambda at
    the bar; FP32 CG needs more iterations there (loss of orthogonality), bounded by 1.5x."""
    p = _probs([(40, 5, 0)], config=65)[0]
    for kind in ("sym", "add", "bj"):
        _, _, x, it_o, _, _, st_o = block.solve_problem(p, kind, 1e-6)
        lam, it, rr, st = gpu_solve_qp_f64(p, kind, 1e-6)
        assert st == 0 and iters_ok(it, it_o, unknowns=p.n * p.nx) and rel(lam, x) <= 1e-7
        lam, it, rr, st = gpu_solve_qp(p, kind, 1e-6)
        assert st == 0 and rr <= 1e-6 and it_o - 1 <= it <= 1.5 * it_o
        assert rel(lam, x) <= LAMBDA_RTOL
