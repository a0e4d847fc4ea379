"""Polynomial (Neumann) preconditioners, Eq. polynomial_precon: the PCG with
Phi_d^-1 = sum_{j<=d} (I - Phi^-1 S)^j Phi^-1 on the GPU against the FP64
oracle applying the same series term by term, through every entry point and
kernel variant that takes the option (batched pipeline with its FP64 subset,
single QP-form and block-form solves, vectors in a global workspace, the
allocation-free solve)."""
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
    from _gpu_helpers import LAMBDA_RTOL, dev, gpu_precond, gpu_solve_qp, is_tiny, iters_match, iters_ok, oracle_blocks32, rel


def _ragged():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=60)
    probs += P.custom_problems([(0, 3, 2), (1, 1, 1), (5, 28, 14), (12, 9, 0), (2, 17, 9)], config=64)
    return probs


def _plan(probs, **kw):
    return sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(**kw))


@pytest.mark.parametrize("kind,degree", [("sym", 1), ("sym", 2), ("sym", 3), ("bj", 1), ("add", 2)])
def test_pipeline_polynomial_matches_oracle(kind, degree):
    probs = _ragged()
    plan = _plan(probs, tol=1e-6, poly_degree=degree)
    b = sspcg.Batch(plan, probs)
    b.pipeline(kind)
    torch.cuda.synchronize()
    xs, it_o, _, st_o, _, _ = block.solve_batch(probs, kind, 1e-6, degree=degree)
    lams = b.lambdas()
    it = b.iters.cpu().numpy(); st = b.status.cpu().numpy(); rr = b.relres.cpu().numpy()
    assert (st == 0).all() and (st_o == 0).all() and (rr <= 1e-6).all()
    for i, p in enumerate(probs):
        assert iters_match(it[i], it_o[i], p, kind), (i, p.N, p.nx, it[i], it_o[i])
        assert rel(lams[i], xs[i]) <= LAMBDA_RTOL, (i, rel(lams[i], xs[i]))


def test_higher_degree_takes_fewer_iterations():
    """On the ragged batch every degree-1 solve takes fewer iterations than degree 0, and the symmetric
    stair at degree d matches block-Jacobi at degree 2d+1 (the same polynomial in D^-1 S)."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=40)
    its = {}
    for kind, d in (("sym", 0), ("sym", 1), ("bj", 3)):
        plan = _plan(probs, tol=1e-6, poly_degree=d)
        b = sspcg.Batch(plan, probs)
        b.pipeline(kind)
        torch.cuda.synchronize()
        assert (b.status.cpu().numpy() == 0).all()
        its[(kind, d)] = b.iters.cpu().numpy()
    assert (its[("sym", 1)] < its[("sym", 0)]).all()
    # the same polynomial, assembled differently: equal up to FP32 rounding of the iteration
    diff = np.abs(its[("sym", 1)] - its[("bj", 3)])
    assert diff.max() <= 2 and diff.mean() <= 0.5


@pytest.mark.parametrize("degree", [1, 2])
def test_single_solves_qp_and_block_form(degree):
    p = P.make_workload(P.MANIPULATOR_SINGLE, count=1)[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym")
    x_o, it_o, _, _, st_o = block.pcg(S, M, p.gamma, 1e-6, degree=degree)
    lam, it, rr, st = gpu_solve_qp(p, "sym", 1e-6, poly_degree=degree)
    assert st == 0 and st_o == 0 and rr <= 1e-6
    assert iters_ok(it, it_o) and rel(lam, x_o) <= LAMBDA_RTOL
    # block form on the oracle's blocks rounded to FP32, against the oracle on the same blocks
    p = P.make_workload(P.RAGGED_BATCH_4096, count=4)[3]
    D32, E32, Sb = oracle_blocks32(p)
    D, E = dev(D32.ravel()), dev(E32.ravel())
    PD, PE, pst = gpu_precond(p, D, E, "sym")
    assert pst == 0
    Mb = block.build_precond(Sb, "sym")
    xb_o, itb_o, _, _, _ = block.pcg(Sb, Mb, p.gamma, 1e-6, degree=degree)
    g = dev(p.gamma)
    lb = torch.zeros_like(g)
    it_t = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    st_t = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve(p.N, p.nx, D, E, PD, PE, g, lb, sspcg.options(tol=1e-6, poly_degree=degree), it_t, rr_t, st_t)
    torch.cuda.synchronize()
    assert int(st_t.item()) == 0
    assert iters_ok(int(it_t.item()), itb_o)
    assert rel(lb.cpu().numpy()[:p.gamma.size].reshape(p.gamma.shape), xb_o) <= LAMBDA_RTOL


def test_global_workspace_vectors_with_polynomial():
    """Problems whose vectors (with the polynomial's extra vector) exceed shared memory."""
    probs = P.custom_problems([(512, 28, 14), (480, 27, 14), (40, 6, 3)], config=65)
    plan = _plan(probs, tol=1e-6, poly_degree=1)
    assert sspcg.sspcg_plan_stats(plan)["pipeline_stream"] >= 2
    b = sspcg.Batch(plan, probs)
    b.pipeline("sym")
    torch.cuda.synchronize()
    xs, it_o, _, _, _, _ = block.solve_batch(probs, "sym", 1e-6, degree=1)
    lams = b.lambdas()
    it = b.iters.cpu().numpy()
    assert (b.status.cpu().numpy() == 0).all()
    for i, p in enumerate(probs):
        assert iters_ok(it[i], it_o[i]), (i, it[i], it_o[i])
        assert rel(lams[i], xs[i]) <= LAMBDA_RTOL


def test_noalloc_solve_with_polynomial():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=48)
    opts = sspcg.options(tol=1e-6, poly_degree=2)
    plan = _plan(probs, tol=1e-6, poly_degree=2)
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
    xs, it_o, _, _, _, _ = block.solve_batch(probs, "sym", 1e-6, degree=2)
    got = plan.unpack(sspcg.ARRAY_VEC, lam, [p.gamma.shape for p in probs])
    itn = it.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    for i, p in enumerate(probs):
        # every problem runs in FP32 here: iteration counts compared above 192 unknowns
        assert is_tiny(p) or iters_match(itn[i], it_o[i], p), (i, itn[i], it_o[i])
        assert rel(got[i], xs[i]) <= LAMBDA_RTOL
