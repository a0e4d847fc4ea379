"""Single-reduction (Chronopoulos-Gear) PCG: the same iterates as the
textbook algorithm the oracle runs, with one block sum per iteration.  The
GPU results are compared with the FP64 textbook oracle (lambda and iteration
counts) through the batched pipeline with its FP64 subset, the single
QP-form solve, vectors in a global workspace, warm starts and the
allocation-free solve."""
import numpy as np
import pytest
import torch

from oracle import block
from paper_2309_06427_gb300 import problems as P

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2309_06427_gb300 import build as _build
    _build.build()
    from paper_2309_06427_gb300 import sspcg
    from _gpu_helpers import LAMBDA_RTOL, gpu_solve_qp, is_tiny, iters_match, iters_ok, rel


def _plan(probs, **kw):
    return sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(cg_variant=1, **kw))


def _check(probs, lams, it, st, rr, tol, kind="sym", all_fp32=False, degree=0):
    """all_fp32: every problem ran in FP32, so the iteration counts of problems of at most 192 unknowns are not
    compared (FP32 CG does not reach the finite termination FP64 CG reaches there; the pipeline runs them in
    FP64)."""
    xs, it_o, _, st_o, _, _ = block.solve_batch(probs, kind, tol, degree=degree)
    assert (st == 0).all() and (st_o == 0).all() and (rr <= tol).all()
    for i, p in enumerate(probs):
        if not (all_fp32 and is_tiny(p)):
            ok = iters_match(it[i], it_o[i], p, kind, tol) if degree == 0 else abs(int(it[i]) - int(it_o[i])) <= 1
            assert ok, (i, p.N, p.nx, it[i], it_o[i])
        assert rel(lams[i], xs[i]) <= LAMBDA_RTOL, (i, rel(lams[i], xs[i]))


@pytest.mark.parametrize("kind", ["sym", "add", "bj"])
def test_pipeline_single_reduction_matches_oracle(kind):
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=64)
    probs += P.custom_problems([(0, 3, 2), (1, 1, 1), (5, 28, 14), (12, 9, 0), (2, 17, 9), (140, 21, 11)],
                               config=86)
    plan = _plan(probs, tol=1e-6)
    b = sspcg.Batch(plan, probs)
    b.pipeline(kind)
    torch.cuda.synchronize()
    _check(probs, b.lambdas(), b.iters.cpu().numpy(), b.status.cpu().numpy(), b.relres.cpu().numpy(), 1e-6, kind)


def test_textbook_and_single_reduction_agree_on_the_ragged_batch():
    """Both variants on 512 problems: iterations within one of each other, lambda within the parity bar."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=512)
    out = []
    for cg in (0, 1):
        plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                       sspcg.options(tol=1e-6, cg_variant=cg))
        b = sspcg.Batch(plan, probs)
        b.pipeline("sym")
        torch.cuda.synchronize()
        assert (b.status.cpu().numpy() == 0).all()
        out.append((b.lambdas(), b.iters.cpu().numpy()))
    assert np.abs(out[0][1] - out[1][1]).max() <= 1
    assert max(rel(out[1][0][i], out[0][0][i]) for i in range(len(probs))) <= LAMBDA_RTOL


def test_single_solve_manipulator_and_maxiter():
    p = P.make_workload(P.MANIPULATOR_SINGLE, count=1)[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym")
    x_o, it_o, _, _, _ = block.pcg(S, M, p.gamma, 1e-6)
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6, cg_variant=1)
    assert st == 0 and rr <= 1e-6 and iters_ok(it, it_o) and rel(lam, x_o) <= LAMBDA_RTOL
    # max_iter: the iterate after exactly 20 x updates, as the textbook oracle's
    x20, it20, _, _, st20 = block.pcg(S, M, p.gamma, 1e-6, max_iter=20)
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6, cg_variant=1, max_iter=20)
    assert it == it20 == 20 and st == sspcg.SOLVE_MAXITER and st20 == block.MAXITER
    assert rel(lam, x20) <= 1e-4


def test_global_workspace_and_warm_start():
    probs = P.custom_problems([(512, 28, 14), (300, 25, 13), (40, 6, 3)], config=87)
    plan = _plan(probs, tol=1e-6, warm_start=2)
    b = sspcg.Batch(plan, probs)
    assert sspcg.sspcg_plan_stats(plan)["pipeline_stream"] >= 2
    b.lam.zero_()
    b.pipeline("sym")
    torch.cuda.synchronize()
    it0 = b.iters.cpu().numpy().copy()
    _check(probs, b.lambdas(), it0, b.status.cpu().numpy(), b.relres.cpu().numpy(), 1e-6)
    # warm re-solve from the solution: far fewer iterations (the FP32 true residual sits near the tolerance)
    d = b.dev
    sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, d["gamma"], b.lam, b.iters,
                                 b.relres, b.status)
    torch.cuda.synchronize()
    assert (b.status.cpu().numpy() == 0).all() and (b.iters.cpu().numpy() <= 0.5 * it0).all()


def test_noalloc_single_reduction():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=40)
    opts = sspcg.options(tol=1e-6, cg_variant=1)
    plan = _plan(probs, tol=1e-6)
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E)
    st0 = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond_batched(plan, "sym", b.D, b.E, b.PD, b.PE, st0)
    lam = plan.empty(sspcg.ARRAY_VEC)
    it = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    rr = torch.zeros(plan.nprob, dtype=torch.float64, device="cuda")
    st = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve_qp_batched_noalloc([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                         d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, d["gamma"], lam, opts, it,
                                         rr, st)
    torch.cuda.synchronize()
    lams = plan.unpack(sspcg.ARRAY_VEC, lam, [p.gamma.shape for p in probs])
    _check(probs, lams, it.cpu().numpy(), st.cpu().numpy(), rr.cpu().numpy(), 1e-6, all_fp32=True)


@pytest.mark.parametrize("kind,degree", [("bj", 1), ("sym", 1), ("bj", 2)])
def test_single_reduction_with_polynomial_preconditioners(kind, degree):
    """Single-reduction PCG with Phi_d^-1 (Horner correction form): block-Jacobi at degree 1 applies the
    symmetric stair implicitly (2 D^-1 - D^-1 S D^-1), reading no off-diagonal preconditioner blocks (the
    pipeline passes none for block-Jacobi).  Against the oracle's textbook PCG with the same series."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=48)
    probs += P.custom_problems([(140, 21, 11), (0, 3, 2), (200, 9, 5)], config=89)
    plan = _plan(probs, tol=1e-6, poly_degree=degree)
    b = sspcg.Batch(plan, probs)
    b.pipeline(kind)
    torch.cuda.synchronize()
    _check(probs, b.lambdas(), b.iters.cpu().numpy(), b.status.cpu().numpy(), b.relres.cpu().numpy(), 1e-6, kind,
           degree=degree)
    if kind == "bj" and degree == 1:
        # the same iterations as the explicit symmetric stair (Sec. IV identity), within the parity bar
        xs, it_sym, _, _, _, _ = block.solve_batch(probs, "sym", 1e-6)
        it = b.iters.cpu().numpy()
        assert all(iters_match(it[i], it_sym[i], p) for i, p in enumerate(probs) if not is_tiny(p))


def test_block_diagonal_preconditioner_without_PE():
    """PE = NULL (block-diagonal preconditioner) gives the same result as passing the zero off-diagonal blocks
    of block-Jacobi, bit for bit."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=32)
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E)
    st0 = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond_batched(plan, "bj", b.D, b.E, b.PD, b.PE, st0)
    outs = []
    for pe in (b.PE, None):
        lam = plan.empty(sspcg.ARRAY_VEC)
        it = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
        rr = torch.zeros(plan.nprob, dtype=torch.float64, device="cuda")
        st = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, pe, d["gamma"], lam, it, rr, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        outs.append((lam.cpu(), it.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
