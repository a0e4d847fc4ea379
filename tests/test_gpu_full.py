"""Full SPD cost blocks Q_k, R_k (Sec. II-A with matrix inverses): the GPU
Schur build against the FP64 oracle, single and batched, NOT-SPD reporting,
and the block-form solve on the resulting blocks against the oracle."""
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
    from _gpu_helpers import LAMBDA_RTOL, dev, is_tiny, iters_match, rel

BLOCK_RTOL = 1e-6
SHAPES = [(0, 3, 2), (1, 1, 1), (4, 3, 2), (7, 5, 0), (12, 9, 5), (20, 28, 14), (33, 17, 9), (64, 14, 7)]


def _probs():
    return P.custom_problems(SHAPES, config=83)


def _gpu_full_single(p, Q, R):
    n, m = p.n, p.nx
    D = torch.zeros(max(n * m * m, 4), device="cuda")
    E = torch.zeros(max(p.N * m * m, 4), device="cuda")
    work = torch.zeros(max(sspcg.sspcg_schur_full_work_floats(p.N, m, p.nu), 4), device="cuda")
    st = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_schur_full(p.N, m, p.nu, dev(p.A), dev(p.B), dev(Q), dev(R), D, E, work, st)
    torch.cuda.synchronize()
    return D, E, int(st.item())


def _check_blocks(p, D, E, S):
    n, m = p.n, p.nx
    Dg = D.cpu().numpy()[:n * m * m].reshape(n, m, m)
    assert np.array_equal(Dg, np.transpose(Dg, (0, 2, 1)))
    assert rel(Dg, S.d) <= BLOCK_RTOL
    if p.N:
        Eg = E.cpu().numpy()[:p.N * m * m].reshape(p.N, m, m)
        assert rel(Eg, S.l[1:]) <= BLOCK_RTOL


@pytest.mark.parametrize("p", _probs(), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_single_full_build_matches_oracle(p):
    Q, R = P.full_cost(p)
    D, E, st = _gpu_full_single(p, Q, R)
    assert st == 0
    _check_blocks(p, D, E, block.build_schur_full(p.A, p.B, Q, R))


def test_diagonal_full_build_matches_diagonal_build():
    """Diagonal Q, R through the full-cost build equal the diagonal build's blocks to FP32 rounding."""
    for p in _probs():
        Q = np.stack([np.diag(q) for q in p.qd]).astype(np.float32)
        R = (np.stack([np.diag(r) for r in p.rd]) if p.N else np.zeros((0, p.nu, p.nu))).astype(np.float32)
        D, E, st = _gpu_full_single(p, Q, R)
        assert st == 0
        _check_blocks(p, D, E, block.build_schur(p.A, p.B, p.qd, p.rd))


def _batched(probs, Qs, Rs, status_init=0):
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, probs)
    Qd = torch.from_numpy(plan.pack(sspcg.ARRAY_DIAG, Qs)).cuda()
    Rd = torch.from_numpy(plan.pack(sspcg.ARRAY_RFULL, Rs)).cuda()
    st = torch.full((plan.nprob,), status_init, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_schur_full_batched(plan, b.dev["A"], b.dev["B"], Qd, Rd, b.D, b.E, st)
    torch.cuda.synchronize()
    return plan, b, st.cpu().numpy()


def test_batched_full_build_and_solve_match_oracle():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=48) + _probs()
    QR = [P.full_cost(p) for p in probs]
    plan, b, st = _batched(probs, [q for q, _ in QR], [r for _, r in QR], status_init=9)
    assert (st == 0).all()
    n_all = plan.sizes
    off_d, off_e = plan.offsets[sspcg.ARRAY_DIAG], plan.offsets[sspcg.ARRAY_OFF]
    Dh, Eh = b.D.cpu().numpy(), b.E.cpu().numpy()
    for i, p in enumerate(probs):
        S = block.build_schur_full(p.A, p.B, *QR[i])
        m = p.nx
        Dg = torch.from_numpy(Dh[off_d[i]:off_d[i] + p.n * m * m].copy())
        Eg = torch.from_numpy(Eh[off_e[i]:off_e[i] + max(p.N * m * m, 0)].copy())
        _check_blocks(p, Dg, Eg if p.N else torch.zeros(4), S)
    assert n_all[sspcg.ARRAY_RFULL] == sum((p.N * p.nu * p.nu + 3) // 4 * 4 for p in probs)
    # block-form solve (problems whose vectors fit in shared memory) on the oracle's full-cost blocks rounded
    # to FP32 on the host, against the oracle's PCG on the same FP32 blocks
    So32 = []
    for i, p in enumerate(probs):
        S = block.build_schur_full(p.A, p.B, *QR[i])
        d = S.d.astype(np.float32).astype(np.float64)
        l = np.zeros_like(d); u = np.zeros_like(d)
        if p.N:
            l[1:] = S.l[1:].astype(np.float32)
            u[:-1] = np.transpose(l[1:], (0, 2, 1))
        So32.append(block.BlockTridiag(d, l, u))
    D32 = torch.from_numpy(plan.pack(sspcg.ARRAY_DIAG, [S.d.astype(np.float32) for S in So32])).cuda()
    E32 = torch.from_numpy(plan.pack(sspcg.ARRAY_OFF, [S.l[1:].astype(np.float32) for S in So32])).cuda()
    stp = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond_batched(plan, "sym", D32, E32, b.PD, b.PE, stp)
    lam = plan.empty(sspcg.ARRAY_VEC)
    it = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    rr = torch.zeros(plan.nprob, dtype=torch.float64, device="cuda")
    sts = torch.zeros(plan.nprob, dtype=torch.int32, device="cuda")
    sspcg.sspcg_solve_batched(plan, D32, E32, b.PD, b.PE, b.dev["gamma"], lam, it, rr, sts)
    torch.cuda.synchronize()
    assert (stp.cpu().numpy() == 0).all() and (sts.cpu().numpy() == 0).all()
    lams = plan.unpack(sspcg.ARRAY_VEC, lam, [p.gamma.shape for p in probs])
    itn = it.cpu().numpy()
    for i, p in enumerate(probs):
        x, it_o, _, _, st_o = block.pcg(So32[i], block.build_precond(So32[i], "sym"), p.gamma, 1e-6)
        # FP32 block form: iteration counts compared above 192 unknowns (FP64 finite termination below)
        assert st_o == 0 and (is_tiny(p) or iters_match(itn[i], it_o, p, S=So32[i])), (i, itn[i], it_o)
        assert rel(lams[i], x) <= LAMBDA_RTOL, (i, rel(lams[i], x))
        # against the FP64 system itself: the true residual of the FP32-block solution
        Sf = block.build_schur_full(p.A, p.B, *QR[i]).dense()
        g = p.gamma.astype(np.float64).ravel()
        assert np.linalg.norm(g - Sf @ lams[i].astype(np.float64).ravel()) <= 1e-4 * np.linalg.norm(g)


def test_indefinite_cost_blocks_are_reported_per_problem():
    probs = P.custom_problems([(6, 4, 2), (5, 3, 2), (8, 5, 3)], config=84)
    QR = [P.full_cost(p) for p in probs]
    Qs = [q.copy() for q, _ in QR]
    Rs = [r.copy() for _, r in QR]
    Qs[0][3] = -Qs[0][3]          # problem 0: an indefinite Q_3
    Rs[2][1][0, 0] = -5.0         # problem 2: an indefinite R_1
    _, _, st = _batched(probs, Qs, Rs)
    assert st.tolist() == [sspcg.SOLVE_NOT_SPD, 0, sspcg.SOLVE_NOT_SPD]
    p = probs[0]
    _, _, st1 = _gpu_full_single(p, Qs[0], Rs[0])
    assert st1 == sspcg.SOLVE_NOT_SPD
