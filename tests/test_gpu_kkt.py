"""The QP step around the solve on the GPU (gamma formation, delta z recovery) against the
dense FP64 definitions, singly and batched, and the whole step against a dense KKT solve."""
import dataclasses

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
    from _gpu_helpers import LAMBDA_RTOL, dev, rel

SHAPES = [(6, 3, 2), (9, 14, 7), (4, 4, 0), (0, 3, 2), (25, 21, 11), (1, 1, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_form_gamma_and_recover_step_match_definitions(shape):
    p = P.custom_problems([shape], config=76)[0]
    c, q, r = P.qp_vectors(p, seed=2)
    n, m = p.n, p.nx
    g = torch.zeros(max(n * m, 4), device="cuda")
    A, B, qd, rd = dev(p.A), dev(p.B), dev(p.qd), dev(p.rd)
    sspcg.sspcg_form_gamma(p.N, m, p.nu, A, B, qd, rd, dev(c), dev(q), dev(r), g)
    mu = np.random.default_rng(4).standard_normal((n, m)).astype(np.float32)
    dx = torch.zeros(max(n * m, 4), device="cuda"); du = torch.zeros(max(p.N * p.nu, 4), device="cuda")
    sspcg.sspcg_recover_step(p.N, m, p.nu, A, B, qd, rd, dev(q), dev(r), dev(mu), dx, du)
    torch.cuda.synchronize()
    g_ref = dense.form_gamma(p.A, p.B, p.qd, p.rd, c, q, r)
    dx_ref, du_ref = dense.recover_step(p.A, p.B, p.qd, p.rd, q, r, mu)
    # FP32 sums of at most 2 * 28 products of FP32 inputs
    assert rel(g.cpu().numpy()[:n * m], g_ref) <= 1e-6
    assert rel(dx.cpu().numpy()[:n * m], dx_ref) <= 1e-6
    if p.N * p.nu:
        assert rel(du.cpu().numpy()[:p.N * p.nu], du_ref) <= 1e-6


def test_batched_qp_step_reaches_the_kkt_solution():
    """gamma on the GPU -> symmetric stair PCG pipeline -> delta z on the GPU, against one dense solve of
    the whole KKT system.  Bound: |dz - dz*| <= |G^-1 C^T| |mu - mu*|, with the PCG bar on mu."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=24) + P.custom_problems(SHAPES, config=77)
    vecs = [P.qp_vectors(p, seed=5) for p in probs]
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    cv = torch.from_numpy(plan.pack(sspcg.ARRAY_VEC, [v[0] for v in vecs])).cuda()
    qv = torch.from_numpy(plan.pack(sspcg.ARRAY_VEC, [v[1] for v in vecs])).cuda()
    rv = torch.from_numpy(plan.pack(sspcg.ARRAY_RD, [v[2] for v in vecs],
                                    np.ones(max(int(plan.sizes[sspcg.ARRAY_RD]), 4), np.float32))).cuda()
    gam = plan.empty(sspcg.ARRAY_VEC)
    sspcg.sspcg_form_gamma_batched(plan, d["A"], d["B"], d["qd"], d["rd"], cv, qv, rv, gam)
    sspcg.sspcg_pipeline_batched(plan, "sym", d["A"], d["B"], d["qd"], d["rd"], gam, b.D, b.E, b.PD, b.PE, b.lam,
                                 b.iters, b.relres, b.status)
    dx = plan.empty(sspcg.ARRAY_VEC)
    du = plan.empty(sspcg.ARRAY_RD)
    sspcg.sspcg_recover_step_batched(plan, d["A"], d["B"], d["qd"], d["rd"], qv, rv, b.lam, dx, du)
    torch.cuda.synchronize()
    assert (b.status.cpu().numpy() == 0).all()
    dxs = plan.unpack(sspcg.ARRAY_VEC, dx, [p.gamma.shape for p in probs])
    dus = plan.unpack(sspcg.ARRAY_RD, du, [(p.N, p.nu) for p in probs])
    mus = b.lambdas()
    for i, (p, (c, q, r)) in enumerate(zip(probs, vecs)):
        kdx, kdu, klam = dense.kkt_solve(p.A, p.B, p.qd, p.rd, c, q, r)
        assert rel(mus[i], -klam) <= LAMBDA_RTOL, i
        G, C = dense.kkt(p.A, p.B, p.qd, p.rd)
        gain = np.linalg.norm(np.linalg.solve(G, C.T), 2)
        z_gpu = dense._z_vector(dxs[i], dus[i]) if p.N else dxs[i].ravel()
        z_ref = dense._z_vector(kdx, kdu) if p.N else kdx.ravel()
        bound = 2 * gain * LAMBDA_RTOL * np.linalg.norm(klam) + 1e-6 * np.linalg.norm(z_ref)
        assert np.linalg.norm(z_gpu - z_ref) <= bound, (i, np.linalg.norm(z_gpu - z_ref), bound)
