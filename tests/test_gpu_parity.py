"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: Schur and preconditioner blocks within 1e-6 (relative Frobenius norm)
of the oracle's FP64 blocks computed from the same inputs; lambda within
1e-5 (relative 2-norm) of the oracle's lambda; iteration counts within one
of the oracle's (iters_match: within one of the range FP64 PCG itself takes
over reorderings of its sums, where that range is wider than one count).
FP32 iteration counts are not compared on problems of at most 192 unknowns,
which the pipeline solves in FP64 (FP32 CG cannot reproduce the finite
termination that FP64 CG reaches there: Thm. 4.2's few distinct
eigenvalues), nor for scalar Jacobi or nu = 0, whose preconditioned spectra
(kappa 3e2 to 1e4) FP32 rounding perturbs enough to delay CG.
Block-form inputs are the oracle's FP64 blocks rounded to FP32 on the host.
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
    from _gpu_helpers import (ITER_TOL, LAMBDA_RTOL, dev, gpu_precond, gpu_schur, gpu_solve_auto, gpu_solve_qp,
                              gpu_solve_qp_f64, is_tiny, iters_match, oracle_blocks32, rel)

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


def _blocks_dev(p):
    """The oracle's Schur blocks of ``p`` rounded to FP32, on the device, and the oracle's view of them."""
    D32, E32, So = oracle_blocks32(p)
    D = dev(D32.ravel())
    E = dev(E32.ravel()) if p.N else torch.zeros(4, device="cuda")
    return D, E, So


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _probs(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_preconditioner_blocks(p, kind):
    """sspcg_build_precond on FP32 blocks against the oracle's preconditioner of the same FP32 blocks."""
    D, E, So = _blocks_dev(p)
    PD, PE, st = gpu_precond(p, D, E, kind)
    assert st == 0
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
    """sspcg_solve (FP32 block form) on FP32 blocks == oracle PCG on the same blocks."""
    D, E, So = _blocks_dev(p)
    PD, PE, _ = gpu_precond(p, D, E, kind)
    g = dev(p.gamma)
    lam = torch.zeros_like(g)
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve(p.N, p.nx, D, E, PD, PE, g, lam, sspcg.options(tol=1e-6), it, rr, st)
    x, it_o, rr_o, _, st_o = block.pcg(So, block.build_precond(So, kind), p.gamma, 1e-6)
    assert int(st.item()) == 0 and st_o == 0
    if not is_tiny(p) and kind != "jacobi":  # FP32: counts compared for the block preconditioners
        assert iters_match(int(it.item()), it_o, p, kind, S=So), (int(it.item()), it_o)
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
    if is_tiny(p) or kind != "jacobi":  # scalar Jacobi in FP32: lambda only
        assert iters_match(it, it_o, p, kind), (it, it_o)
    assert rel(lam, x) <= LAMBDA_RTOL
    assert rr <= 1e-6


@pytest.mark.parametrize("p", _probs([s for s in SHAPES if (s[0] + 1) * s[1] <= 192]),
                         ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_fp32_path_on_tiny_problems(p):
    """FP32 forced on problems of at most 192 unknowns: lambda at the parity bar.  Their iteration count is
    not compared: FP64 CG ends there by finite termination (few distinct eigenvalues), which FP32 rounding
    does not reproduce; the pipeline solves these problems in FP64."""
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6)
    _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
    assert st == 0 and rr <= 1e-6
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
        # FP32 forced: same answer; more iterations, since FP32 does not reach the finite termination
        lam32, it32, rr32, st32 = gpu_solve_qp(p, kind, 1e-8)
        assert st32 == 0 and rr32 <= 1e-8 and rel(lam32, x) <= LAMBDA_RTOL


@pytest.mark.parametrize("reduction", ["df", "f32", "f64"])
@pytest.mark.parametrize("schedule", ["resident", "stream"])
def test_reduction_modes_and_schedules(reduction, schedule):
    for p in _probs([(64, 14, 7), (30, 21, 11), (5, 3, 2)], h=0.01, config=56):
        lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6, reduction=reduction, schedule=schedule)
        _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
        assert st == 0 and (is_tiny(p) or iters_match(it, it_o, p)), (p.N, p.nx, it, it_o)
        assert rel(lam, x) <= LAMBDA_RTOL


@pytest.mark.parametrize("schedule", ["resident", "stream"])
def test_fp64_path_schedules(schedule):
    for p in _probs([(40, 4, 2), (10, 12, 6), (64, 14, 7)], h=0.01, config=64):
        lam, it, rr, st = gpu_solve_qp_f64(p, "sym", 1e-6, schedule=schedule)
        _, _, x, it_o, _, _, _ = block.solve_problem(p, "sym", 1e-6)
        assert st == 0 and iters_match(it, it_o, p), (it, it_o)
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
    """The FP64 true-residual kernel against the dense definition, for a seeded host-made lambda."""
    p = _probs([(40, 9, 5)], config=62)[0]
    lam = (0.1 * P.normals(P.config_key(62, 7), p.gamma.size)).astype(np.float32).reshape(p.gamma.shape)
    A, B, qd, rd = dev(p.A), dev(p.B), dev(p.qd), dev(p.rd)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sspcg.sspcg_residual_qp(p.N, p.nx, p.nu, A, B, qd, rd, dev(p.gamma), dev(lam), out)
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    g = p.gamma.astype(np.float64).ravel()
    want = np.linalg.norm(g - Sd @ lam.astype(np.float64).ravel()) / np.linalg.norm(g)
    assert abs(out.item() - want) <= 1e-6 * want + 1e-13


def test_inputless_dynamics_nu0():
    """nu = 0 (no inputs, B empty): S = C G^-1 C^T with state rows only, far worse conditioned
    (kappa(S) ~ 9e4, kappa(Phi_sym^-1 S) ~ 3e3 at N = 40, nx = 5).  FP64 path: oracle parity, iterations by
    iters_match (FP64 reorderings alone move the block-Jacobi count over 245..247 here).  FP32 path: lambda
    at the bar and converged; its iteration count is not compared: FP32 rounding perturbs the spectrum CG
    sees by about 2^-24 kappa(Phi^-1 S) ~ 2e-4 relative, which delays convergence (about 30 % here)."""
    p = _probs([(40, 5, 0)], config=65)[0]
    for kind in ("sym", "add", "bj"):
        _, _, x, it_o, _, _, st_o = block.solve_problem(p, kind, 1e-6)
        lam, it, rr, st = gpu_solve_qp_f64(p, kind, 1e-6)
        assert st == 0 and iters_match(it, it_o, p, kind) and rel(lam, x) <= 1e-7, (kind, it, it_o)
        lam, it, rr, st = gpu_solve_qp(p, kind, 1e-6)
        assert st == 0 and rr <= 1e-6
        assert rel(lam, x) <= LAMBDA_RTOL


def _block_solve(p, D32, E32, kind, gamma):
    D = dev(D32.ravel())
    E = dev(E32.ravel()) if p.N else torch.zeros(4, device="cuda")
    PD, PE, pst = gpu_precond(p, D, E, kind)
    g = dev(gamma)
    lam = torch.zeros_like(g)
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve(p.N, p.nx, D, E, PD, PE, g, lam, sspcg.options(tol=1e-6), it, rr, st)
    torch.cuda.synchronize()
    return int(st.item()), int(it.item()), pst


def test_nonfinite_inputs_are_reported():
    """A NaN in gamma (QP form, FP32 and FP64 paths) and a NaN in an operator block (block form, with a
    preconditioner built from finite blocks) end the solve with SSPCG_SOLVE_NONFINITE."""
    p = _probs([(10, 4, 2)], config=67)[0]
    g = p.gamma.copy()
    g[3, 1] = np.nan
    pn = P.Problem(p.N, p.nx, p.nu, p.A, p.B, p.qd, p.rd, g)
    assert gpu_solve_qp(pn, "sym", 1e-6)[3] == sspcg.SOLVE_NONFINITE
    assert gpu_solve_qp_f64(pn, "sym", 1e-6)[3] == sspcg.SOLVE_NONFINITE
    D32, E32, _ = oracle_blocks32(p)
    PD_ok, PE_ok, pst = gpu_precond(p, dev(D32.ravel()), dev(E32.ravel()), "sym")
    assert pst == 0
    Dn = D32.copy()
    Dn[4, 1, 2] = Dn[4, 2, 1] = np.nan
    lam = torch.zeros(p.gamma.size, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve(p.N, p.nx, dev(Dn.ravel()), dev(E32.ravel()), PD_ok, PE_ok, dev(p.gamma), lam,
                      sspcg.options(tol=1e-6), it, rr, st)
    torch.cuda.synchronize()
    assert int(st.item()) == sspcg.SOLVE_NONFINITE


def test_indefinite_operator_breaks_down():
    """An indefinite operator (diagonal blocks I, off-diagonal blocks 2 I) with the block-Jacobi preconditioner
    (the identity) and gamma along its most negative eigenvector: p.Sp < 0 at the first step, so PCG stops
    with SSPCG_SOLVE_BREAKDOWN, as the oracle does."""
    N, nx = 5, 2
    p = P.custom_problems([(N, nx, 1)], config=68)[0]
    D32 = np.tile(np.eye(nx, dtype=np.float32), (N + 1, 1, 1))
    E32 = np.tile(2 * np.eye(nx, dtype=np.float32), (N, 1, 1))
    d = D32.astype(np.float64); l = np.zeros_like(d); u = np.zeros_like(d)
    l[1:] = E32; u[:-1] = E32
    So = block.BlockTridiag(d, l, u)
    w, V = np.linalg.eigh(So.dense())
    assert w[0] < 0
    gamma = V[:, 0].astype(np.float32).reshape(N + 1, nx)
    st, it, pst = _block_solve(p, D32, E32, "bj", gamma)
    _, _, _, _, st_o = block.pcg(So, block.build_precond(So, "bj"), gamma, 1e-6)
    assert pst == 0 and st == sspcg.SOLVE_BREAKDOWN and st_o == block.BREAKDOWN and it == 0
