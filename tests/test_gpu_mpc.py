"""Full-size MPC batch (16,384 problems, N ~ U{64..512}, nx ~ U{4..28}): the whole
path from lambda0 = 0, then sequential re-solves with gamma perturbed by 1 % and
warm-started from the previous solution, in the launch configuration the
benchmark's MPC section times.  Sampled problems against the FP64 oracle; every
problem against its own convergence bar and its FP64 true residual."""
import dataclasses

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
    from _gpu_helpers import LAMBDA_RTOL, iters_match, rel

W = P.MPC_BATCH_16384
RESOLVES = 2


def _oracle_warm(p, x0, tol):
    """Oracle PCG from x0 with the library's fallback rule (start from zero unless ||gamma - S x0|| < ||gamma||)."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    g = p.gamma.astype(np.float64)
    x0 = x0.astype(np.float64)
    y = np.einsum("kij,kj->ki", S.d, x0)
    y[1:] += np.einsum("kij,kj->ki", S.l[1:], x0[:-1])
    y[:-1] += np.einsum("kij,kj->ki", S.u[:-1], x0[1:])
    start = x0 if np.linalg.norm(g - y) < np.linalg.norm(g) else None
    M = block.build_precond(S, "sym")
    return block.pcg(S, M, g, tol, None, start)


def test_mpc_batch_full_size_resolves():
    probs = P.make_workload_parallel(W)
    assert len(probs) == W.nprob
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=W.tol, warm_start=2))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    b.lam.zero_()  # lambda0 = 0: the fallback rule starts the first solve from zero
    b.pipeline("sym")
    torch.cuda.synchronize()
    st, rr, it0 = b.status.cpu().numpy(), b.relres.cpu().numpy(), b.iters.cpu().numpy().copy()
    assert (st == 0).all() and (rr <= W.tol).all()
    rt = torch.zeros(plan.nprob, dtype=torch.float64, device="cuda")
    sspcg.sspcg_residual_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.lam, rt)
    torch.cuda.synchronize()
    assert (rt.cpu().numpy() <= 1e-4).all()
    # 256 problems sampled across the batch against the oracle, one by one
    idx = np.sort(np.random.default_rng(5).choice(len(probs), 256, replace=False))
    sample = [probs[i] for i in idx]
    xs, it_o, _, st_o, _, _ = block.solve_batch(sample, "sym", W.tol)
    assert (st_o == 0).all()
    lams = b.lambdas()
    for j, i in enumerate(idx):
        p = probs[i]
        assert iters_match(it0[i], it_o[j], p), (i, p.N, p.nx, it0[i], it_o[j])
        assert rel(lams[i], xs[j]) <= LAMBDA_RTOL

    # the warm chains: the GPU's from its own previous solutions, the oracle's from its own
    prev_o = {int(i): xs[j] for j, i in enumerate(idx[:64])}
    for r in range(RESOLVES):
        pert = [dataclasses.replace(p, gamma=P.perturb_gamma(p, r)) for p in probs]
        g = torch.from_numpy(plan.pack(sspcg.ARRAY_VEC, [q.gamma for q in pert])).cuda()
        sspcg.sspcg_solve_qp_batched(plan, d["A"], d["B"], d["qd"], d["rd"], b.PD, b.PE, g, b.lam, b.iters, b.relres,
                                     b.status)
        torch.cuda.synchronize()
        it = b.iters.cpu().numpy()
        assert (b.status.cpu().numpy() == 0).all() and (b.relres.cpu().numpy() <= W.tol).all()
        # a 1 % change of gamma leaves most of the previous solution valid
        assert it.mean() < 0.8 * it0.mean(), (r, it.mean(), it0.mean())
        lams = b.lambdas()
        for i in idx[:64]:
            x, it_w, _, _, _ = _oracle_warm(pert[i], prev_o[int(i)], W.tol)
            assert abs(int(it[i]) - it_w) <= 1, (r, i, it[i], it_w)
            assert rel(lams[i], x) <= LAMBDA_RTOL
            prev_o[int(i)] = x
