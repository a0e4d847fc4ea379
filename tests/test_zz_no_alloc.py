"""The allocation-free batched solve (sspcg_solve_qp_batched_noalloc), for
callers that cannot call cudaMalloc once running (a real-time control loop,
an application whose allocator owns the device memory).  Its results must
match the plan-based sspcg_solve_qp_batched on the same inputs, on two calls
in a row (the calls share one file-scope scratch array)."""
import numpy as np
import pytest
import torch

from paper_2309_06427_gb300 import problems as P

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2309_06427_gb300 import build as _build
    _build.build()
    from paper_2309_06427_gb300 import sspcg
    from _gpu_helpers import ITER_TOL, LAMBDA_RTOL, rel


def _batch():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=96)
    probs += P.custom_problems([(0, 3, 2), (1, 1, 1), (5, 28, 14), (12, 9, 0), (130, 21, 11)], config=66)
    return probs


def test_noalloc_solve_matches_plan_solve_twice():
    probs = _batch()
    opts = sspcg.options(tol=1e-6)
    Ns, nxs, nus = [p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs]
    plan = sspcg.sspcg_plan_create(Ns, nxs, nus, opts)
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E)
    st0 = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond_batched(plan, "sym", b.D, b.E, b.PD, b.PE, st0)
    ref_lam = plan.empty(sspcg.ARRAY_VEC)
    ref_it = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    ref_rr = torch.zeros(plan.nprob, dtype=torch.float64, device="cuda")
    ref_st = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, d["gamma"], ref_lam, ref_it,
                                 ref_rr, ref_st)
    torch.cuda.synchronize()
    assert (ref_st.cpu().numpy() == 0).all()
    shapes = [p.gamma.shape for p in probs]
    ref = plan.unpack(sspcg.ARRAY_VEC, ref_lam, shapes)
    outs = [(plan.empty(sspcg.ARRAY_VEC, fill=float("nan")),
             torch.full((plan.nprob,), -7, dtype=torch.int32, device="cuda"),
             torch.zeros(plan.nprob, dtype=torch.float64, device="cuda"),
             torch.full((plan.nprob,), 9, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        lam, it, rr, st = outs[call]
        free_before = torch.cuda.mem_get_info()[0]
        sspcg.sspcg_solve_qp_batched_noalloc(Ns, nxs, nus, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE,
                                             d["gamma"], lam, opts, it, rr, st)
        torch.cuda.synchronize()
        # the call takes no device memory: free bytes are the same after it
        assert torch.cuda.mem_get_info()[0] == free_before, call
        assert (st.cpu().numpy() == 0).all(), call
        assert np.abs(it.cpu().numpy() - ref_it.cpu().numpy()).max() <= ITER_TOL, call
        got = plan.unpack(sspcg.ARRAY_VEC, lam, shapes)
        assert max(rel(got[i], ref[i]) for i in range(len(probs))) <= LAMBDA_RTOL, call
        assert (rr.cpu().numpy() <= 1e-6).all()


def test_noalloc_rejects_batches_beyond_its_scratch():
    n = sspcg.NOALLOC_MAX_PROBLEMS + 1
    z = torch.zeros(4, device="cuda")
    zi = torch.zeros(4, dtype=torch.int32, device="cuda")
    zd = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(sspcg.SspcgError, match="invalid argument"):
        sspcg.sspcg_solve_qp_batched_noalloc([4] * n, [2] * n, [1] * n, z, z, z, z, z, z, z, z,
                                             sspcg.options(), zi, zd, zi)


def test_noalloc_call_replays_from_a_cuda_graph():
    """After a first call (the warm-up the header asks for), the allocation-free solve can be captured into a
    CUDA graph: it copies nothing from host memory (the shapes travel as a set-up kernel's parameters), so each
    replay solves the captured batch again, bit-identical to the direct call."""
    probs = _batch()
    opts = sspcg.options(tol=1e-6)
    Ns, nxs, nus = [p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs]
    plan = sspcg.sspcg_plan_create(Ns, nxs, nus, opts)
    b = sspcg.Batch(plan, probs)
    d = b.dev
    sspcg.sspcg_build_schur_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.D, b.E)
    st0 = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond_batched(plan, "sym", b.D, b.E, b.PD, b.PE, st0)

    def outputs():  # lambda prefilled with a finite sentinel: the padding between problems is never written
        return (plan.empty(sspcg.ARRAY_VEC, fill=123.0),
                torch.full((plan.nprob,), -7, dtype=torch.int32, device="cuda"),
                torch.zeros(plan.nprob, dtype=torch.float64, device="cuda"),
                torch.full((plan.nprob,), 9, dtype=torch.int32, device="cuda"))

    def call(o):
        sspcg.sspcg_solve_qp_batched_noalloc(Ns, nxs, nus, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE,
                                             d["gamma"], o[0], opts, o[1], o[2], o[3])

    direct = outputs()
    call(direct)  # also the warm-up
    torch.cuda.synchronize()
    assert (direct[3].cpu().numpy() == 0).all()
    cap = outputs()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call(cap)
    torch.cuda.synchronize()
    for rep in range(2):
        cap[0].fill_(123.0); cap[1].fill_(-7); cap[3].fill_(9)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(cap[0], direct[0]), rep
        assert torch.equal(cap[1], direct[1]) and torch.equal(cap[2], direct[2]), rep
        assert (cap[3].cpu().numpy() == 0).all(), rep
