"""Learned warm start on the GPU against the FP64 oracle (oracle/mlp.py): knot
features, normalisation, forward pass, gradients of one training step, the Adam
update, and what the trained network gains over the plain start."""
import numpy as np
import pytest
import torch

from oracle import block
from oracle import mlp as omlp
from paper_2309_06427_gb300 import problems as P

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2309_06427_gb300 import build as _build
    _build.build()
    from paper_2309_06427_gb300 import sspcg
    from _gpu_helpers import LAMBDA_RTOL, rel

BF16_ULP = 2.0 ** -8  # half-ulp relative step of bfloat16 (7 fraction bits)


def _problems():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=10)
    probs += P.custom_problems([(0, 3, 2), (5, 28, 14), (4, 6, 0), (9, 2, 1), (3, 21, 11)], config=72)
    return probs


def _setup(probs, max_rows=4096):
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, probs)
    b.pipeline("sym")
    torch.cuda.synchronize()
    net = sspcg.sspcg_mlp_create(max_rows)
    return plan, b, net


def _oracle_features(probs):
    Ss = [block.build_schur(p.A, p.B, p.qd, p.rd) for p in probs]
    return Ss, np.concatenate([omlp.knot_features(p, S) for p, S in zip(probs, Ss)])


def _random_params(seed):
    prm = P.mlp_initial_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    o = omlp.unflatten(prm)
    o["W3"] = rng.standard_normal(o["W3"].shape) * 0.05
    o["b1"] = rng.standard_normal(256) * 0.05
    o["b2"] = rng.standard_normal(256) * 0.05
    o["b3"] = rng.standard_normal(32) * 0.05
    flat32 = omlp.flatten(o).astype(np.float32)
    return flat32, omlp.unflatten(flat32.astype(np.float64))


def _set_norm(net, mu, isd):
    mu32, isd32 = mu.astype(np.float32), isd.astype(np.float32)
    sspcg.sspcg_mlp_set_normalisation(net, torch.from_numpy(mu32).cuda(), torch.from_numpy(isd32).cuda())
    return mu32.astype(np.float64), isd32.astype(np.float64)


def _gpu_features(net, plan, b, p0, p1, rows):
    X = torch.zeros((rows, sspcg.MLP_IN), dtype=torch.bfloat16, device="cuda")
    d = b.dev
    sspcg.sspcg_mlp_features(net, plan, p0, p1, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, X)
    torch.cuda.synchronize()
    return X.float().cpu().numpy().astype(np.float64)


def test_features_match_oracle():
    probs = _problems()
    plan, b, net = _setup(probs)
    _, F = _oracle_features(probs)
    Xg = _gpu_features(net, plan, b, 0, len(probs), F.shape[0])  # normalisation mu = 0, 1/sigma = 1
    Xo = omlp.bf16_round(F)
    dj = np.zeros(omlp.D_IN, bool); dj[omlp.OFF_DJ:omlp.OFF_DJ + 28] = True
    # every column but D^-1 gamma is an FP32 input rounded to bfloat16 the same way on both sides
    assert np.array_equal(Xg[:, ~dj], Xo[:, ~dj])
    # D^-1 gamma: FP32 preconditioner blocks against an FP64 solve, then bfloat16 (one step at most)
    err = np.abs(Xg[:, dj] - Xo[:, dj])
    assert (err <= 2 * BF16_ULP * np.abs(Xo[:, dj]) + 1e-6).all()
    # a sub-range of problems gives the same rows
    ks = np.cumsum([0] + [p.n for p in probs])
    Xs = _gpu_features(net, plan, b, 3, 7, ks[7] - ks[3])
    assert np.array_equal(Xs, Xg[ks[3]:ks[7]])


def test_normalisation_fit_matches_oracle():
    probs = _problems()
    plan, b, net = _setup(probs)
    _, F = _oracle_features(probs)
    mu_o, isd_o = omlp.normalisation(F)
    d = b.dev
    sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)
    mu = torch.zeros(omlp.D_IN, device="cuda"); isd = torch.zeros(omlp.D_IN, device="cuda")
    sspcg.sspcg_mlp_get_normalisation(net, mu, isd)
    torch.cuda.synchronize()
    mu, isd = mu.cpu().numpy(), isd.cpu().numpy()
    assert np.array_equal(isd == 0, isd_o == 0)
    assert np.allclose(mu, mu_o, rtol=1e-5, atol=1e-6)
    live = isd_o > 0
    assert np.allclose(isd[live], isd_o[live], rtol=1e-4)


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_forward_matches_oracle(engine):
    probs = _problems()
    plan, b, net = _setup(probs)
    sspcg.sspcg_mlp_set_engine(net, engine)
    Ss, F = _oracle_features(probs)
    mu, isd = _set_norm(net, *omlp.normalisation(F))
    flat32, prm = _random_params(7)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(flat32).cuda())
    lam0 = plan.empty(sspcg.ARRAY_VEC)
    d = b.dev
    sspcg.sspcg_mlp_infer(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, lam0)
    torch.cuda.synchronize()
    got = plan.unpack(sspcg.ARRAY_VEC, lam0, [p.gamma.shape for p in probs])
    X = omlp.normalise(F, mu, isd)
    ref = omlp.warm_start(prm, X, [p.nx for p in probs], [p.n for p in probs])
    # FP32 accumulation order and rare bfloat16 rounding flips of hidden activations
    for g, r in zip(got, ref):
        assert rel(g, r) <= 2e-3
    assert rel(np.concatenate([g.ravel() for g in got]), np.concatenate([r.ravel() for r in ref])) <= 5e-4
    assert sspcg.sspcg_mlp_status(net) == 0


def test_engines_agree_over_many_tiles_and_chunks():
    """Inference over ~9,000 knot rows in chunks of 1,000 (ragged tails in every 128-row tile grid)."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=120, start=500)
    plan, b, net = _setup(probs, max_rows=1000)
    Ss, F = _oracle_features(probs[:6])
    d = b.dev
    sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)
    flat32, prm = _random_params(3)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(flat32).cuda())
    out = {}
    for engine in ("tcgen05", "mma_sync"):
        sspcg.sspcg_mlp_set_engine(net, engine)
        lam0 = plan.empty(sspcg.ARRAY_VEC)
        sspcg.sspcg_mlp_infer(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, lam0)
        torch.cuda.synchronize()
        out[engine] = lam0.cpu().numpy().astype(np.float64)
    assert sspcg.sspcg_mlp_status(net) == 0
    assert np.isfinite(out["tcgen05"]).all() and np.abs(out["tcgen05"]).max() > 0
    assert rel(out["tcgen05"], out["mma_sync"]) <= 5e-4
    # the first problems against the oracle, with the normalisation the GPU fitted
    mu = torch.zeros(omlp.D_IN, device="cuda"); isd = torch.zeros(omlp.D_IN, device="cuda")
    sspcg.sspcg_mlp_get_normalisation(net, mu, isd)
    torch.cuda.synchronize()
    X = omlp.normalise(F, mu.cpu().numpy().astype(np.float64), isd.cpu().numpy().astype(np.float64))
    ref = omlp.warm_start(prm, X, [p.nx for p in probs[:6]], [p.n for p in probs[:6]])
    got = plan.unpack(sspcg.ARRAY_VEC, torch.from_numpy(out["tcgen05"].astype(np.float32)),
                      [p.gamma.shape for p in probs])[:6]
    assert rel(np.concatenate([g.ravel() for g in got]), np.concatenate([r.ravel() for r in ref])) <= 5e-4


def _train_inputs(probs, b):
    xs, _, _, _, _, _ = block.solve_batch(probs, "sym", 1e-10)
    lam_star = b.plan.pack(sspcg.ARRAY_VEC, [x.astype(np.float32) for x in xs])
    return xs, torch.from_numpy(lam_star).cuda()


def _grad_dict(net):
    g = torch.zeros(sspcg.MLP_PARAMS, device="cuda")
    sspcg.sspcg_mlp_get_grads(net, g)
    torch.cuda.synchronize()
    return omlp.unflatten(g.cpu().numpy().astype(np.float64))


def test_train_step_gradients_match_oracle():
    probs = _problems()
    plan, b, net = _setup(probs)
    Ss, F = _oracle_features(probs)
    mu, isd = _set_norm(net, *omlp.normalisation(F))
    flat32, prm = _random_params(9)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(flat32).cuda())
    xs, lam_star = _train_inputs(probs, b)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = b.dev
    p0, p1 = 2, len(probs)
    sspcg.sspcg_mlp_train_step(net, plan, p0, p1, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E, b.PD,
                               lam_star, sspcg.adam(lr=0.0), loss)
    torch.cuda.synchronize()
    g = _grad_dict(net)
    sub = probs[p0:p1]
    X = omlp.normalise(F[sum(p.n for p in probs[:p0]):], mu, isd)
    cache = omlp.forward(prm, X)
    lam0, o = [], 0
    for p in sub:
        lam0.append(cache["Y"][o:o + p.n, :p.nx]); o += p.n
    L, dl = omlp.loss_and_grad(Ss[p0:p1], lam0, [x.astype(np.float32).astype(np.float64) for x in xs[p0:p1]],
                               [p.gamma for p in sub])
    go = omlp.backward(prm, cache, omlp.output_gradient(dl, [p.nx for p in sub]))
    # FP32 blocks against FP64: u = S(lambda0 - lambda*) cancels to about gamma, so its relative error is
    # about kappa(S) * 2^-24 (up to ~1e-3 on these problems)
    assert abs(loss.item() - L) <= 5e-3 * L
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel(g[name], go[name]) <= 1e-2, name
    # padding outputs 28..31 get no gradient
    assert not g["W3"][28:].any() and not g["b3"][28:].any()


def test_adam_step_matches_oracle():
    probs = _problems()
    plan, b, net = _setup(probs)
    _, F = _oracle_features(probs)
    _set_norm(net, *omlp.normalisation(F))
    flat32, prm = _random_params(4)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(flat32).cuda())
    _, lam_star = _train_inputs(probs, b)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = b.dev
    st = {}
    for step in range(3):
        sspcg.sspcg_mlp_train_step(net, plan, 0, len(probs), d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E,
                                   b.PD, lam_star, sspcg.adam(lr=1e-3), loss)
        torch.cuda.synchronize()
        g = _grad_dict(net)
        omlp.adam(prm, g, st, lr=1e-3)  # the oracle's Adam on the GPU's gradients
        w = torch.zeros(sspcg.MLP_PARAMS, device="cuda")
        sspcg.sspcg_mlp_get_params(net, w)
        torch.cuda.synchronize()
        diff = np.abs(w.cpu().numpy().astype(np.float64) - omlp.flatten(prm))
        assert diff.max() <= 2e-6, (step, diff.max())


def test_invalid_arguments():
    probs = _problems()[:3]
    plan, b, net = _setup(probs, max_rows=8)
    d = b.dev
    X = torch.zeros((4096, sspcg.MLP_IN), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sspcg.SspcgError):  # more rows than the workspace
        sspcg.sspcg_mlp_features(net, plan, 0, 3, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, X)
    with pytest.raises(sspcg.SspcgError):
        sspcg.sspcg_mlp_features(net, plan, 2, 1, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, X)
    with pytest.raises(sspcg.SspcgError):
        sspcg.sspcg_mlp_create(0)


def test_inputs_wider_than_the_feature_layout_are_unsupported():
    """The layout pads B_k to 28 x 14: a batch with nu = 15 is refused on the host, before any kernel."""
    probs = P.custom_problems([(6, 20, 15), (4, 5, 3)], config=85)
    plan = sspcg.sspcg_plan_create([p.N for p in probs], [p.nx for p in probs], [p.nu for p in probs],
                                   sspcg.options(tol=1e-6))
    b = sspcg.Batch(plan, probs)
    d = b.dev
    net = sspcg.sspcg_mlp_create(1024)
    lam0 = plan.empty(sspcg.ARRAY_VEC)
    with pytest.raises(sspcg.SspcgError, match="unsupported"):
        sspcg.sspcg_mlp_infer(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, lam0)
    with pytest.raises(sspcg.SspcgError, match="unsupported"):
        sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)


def _train(net, plan, b, lam_star, epochs, chunk, seed=0):
    """Minibatches of ``chunk`` consecutive problems in a seeded random order; mean loss per epoch."""
    d = b.dev
    starts = list(range(0, plan.nprob, chunk))
    rng = np.random.default_rng(seed)
    loss = torch.zeros(len(starts), dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(epochs):
        for j, s0 in enumerate(rng.permutation(starts)):
            sspcg.sspcg_mlp_train_step(net, plan, int(s0), min(int(s0) + chunk, plan.nprob), d["A"], d["B"], d["qd"],
                                       d["rd"], d["gamma"], b.D, b.E, b.PD, lam_star, sspcg.adam(lr=1e-3), loss[j:j + 1])
        hist.append(float(loss.mean().item()))
    return hist


def test_trained_network_reduces_iterations():
    """Trained on plain solves from the manipulator-like (nx = 14, N = 64, h = 0.01) and ragged-batch generators,
    evaluated on held-out warm-start problems: lower initial residual and fewer PCG iterations than lambda0 = 0,
    with the same solution as the oracle."""
    train = [P.make_problem(P.config_key(2, i), 64, 14, 7, 0.01) for i in range(640)]
    train += P.make_workload(P.RAGGED_BATCH_4096, count=640, start=2000)
    plan, b, net = _setup(train, max_rows=8192)
    assert (b.status.cpu().numpy() == 0).all()
    d = b.dev
    sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)
    sspcg.sspcg_mlp_set_params(net, torch.from_numpy(P.mlp_initial_params(0)).cuda())
    hist = _train(net, plan, b, b.lam.clone(), epochs=8, chunk=32)
    assert abs(hist[0] - 1.0) < 0.2 and hist[-1] < 0.9 * hist[0], hist

    ev = P.make_workload(P.WARMSTART_EVAL_4096, count=192)
    pe = sspcg.sspcg_plan_create([p.N for p in ev], [p.nx for p in ev], [p.nu for p in ev], sspcg.options(tol=1e-6))
    be = sspcg.Batch(pe, ev)
    be.pipeline("sym")
    torch.cuda.synchronize()
    it_plain = be.iters.cpu().numpy().copy()
    de = be.dev
    lam0 = pe.empty(sspcg.ARRAY_VEC)
    sspcg.sspcg_mlp_infer(net, pe, de["A"], de["B"], de["qd"], de["rd"], de["gamma"], be.PD, lam0)
    sspcg.sspcg_pipeline_warm_batched(pe, net, "sym", de["A"], de["B"], de["qd"], de["rd"], de["gamma"], be.D, be.E,
                                      be.PD, be.PE, be.lam, be.iters, be.relres, be.status)
    torch.cuda.synchronize()
    it_warm = be.iters.cpu().numpy()
    assert (be.status.cpu().numpy() == 0).all() and (be.relres.cpu().numpy() <= 1e-6).all()
    l0 = pe.unpack(sspcg.ARRAY_VEC, lam0, [p.gamma.shape for p in ev])
    r0 = []
    for p, x0 in zip(ev[:48], l0[:48]):
        S = block.build_schur(p.A, p.B, p.qd, p.rd)
        g = p.gamma.astype(np.float64)
        r0.append(np.linalg.norm(g - omlp.bt_apply(S, x0.astype(np.float64))) / np.linalg.norm(g))
    print(f"\nwarm start: loss {hist[0]:.3f} -> {hist[-1]:.3f}; held-out ||r0||/||gamma|| mean {np.mean(r0):.3f}; "
          f"PCG iterations plain {it_plain.mean():.2f} warm {it_warm.mean():.2f}")
    assert np.mean(r0) < 0.95
    assert it_warm.mean() < it_plain.mean()
    # the solution does not depend on the start
    xs, _, _, _, _, _ = block.solve_batch(ev[:32], "sym", 1e-6)
    lams = be.lambdas()
    assert max(rel(lams[i], xs[i]) for i in range(32)) <= LAMBDA_RTOL


def test_checkpoint_resumes_training_bit_for_bit():
    """Train k steps, save, load into a fresh network, train k more: the same parameters, Adam moments, step
    count and normalisation, bit for bit, as 2k steps without the interruption."""
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=96)
    plan, b, net_a = _setup(probs)
    d = b.dev
    lam_star = b.lam.clone()
    init = torch.from_numpy(P.mlp_initial_params(3)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    chunks = [(s0, min(s0 + 16, plan.nprob)) for s0 in range(0, plan.nprob, 16)]

    def steps(net, j0, j1):
        for j in range(j0, j1):
            s0, s1 = chunks[(5 * j) % len(chunks)]
            sspcg.sspcg_mlp_train_step(net, plan, s0, s1, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.D, b.E,
                                       b.PD, lam_star, sspcg.adam(lr=1e-3), loss)

    def fresh():
        net = sspcg.sspcg_mlp_create(4096)
        sspcg.sspcg_mlp_fit_normalisation(net, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD)
        sspcg.sspcg_mlp_set_params(net, init)
        return net

    k = 7
    net_a = fresh()
    steps(net_a, 0, 2 * k)
    blob_a = sspcg.sspcg_mlp_save(net_a)
    net_b = fresh()
    steps(net_b, 0, k)
    blob_mid = sspcg.sspcg_mlp_save(net_b)
    del net_b
    net_c = sspcg.sspcg_mlp_create(4096)  # fresh: zero parameters, identity normalisation, no Adam state
    sspcg.sspcg_mlp_load(net_c, blob_mid)
    steps(net_c, k, 2 * k)
    blob_c = sspcg.sspcg_mlp_save(net_c)
    assert blob_a.size == sspcg.sspcg_mlp_checkpoint_bytes()
    assert np.array_equal(blob_a, blob_c)
    assert not np.array_equal(blob_a, blob_mid)
    # the resumed network also infers the same lambda0
    la, lc = plan.empty(sspcg.ARRAY_VEC), plan.empty(sspcg.ARRAY_VEC)
    sspcg.sspcg_mlp_infer(net_a, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, la)
    sspcg.sspcg_mlp_infer(net_c, plan, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], b.PD, lc)
    torch.cuda.synchronize()
    assert torch.equal(la, lc)
    # a blob of another layout is refused
    bad = blob_mid.copy()
    bad[:8] = np.frombuffer(b"NOTMLPCK", dtype=np.uint8)
    with pytest.raises(sspcg.SspcgError, match="invalid argument"):
        sspcg.sspcg_mlp_load(net_c, bad)
    with pytest.raises(sspcg.SspcgError, match="invalid argument"):
        sspcg.sspcg_mlp_load(net_c, blob_mid[:100])
