"""Pins of the warm-start oracle (oracle/mlp.py) against things other than itself:
the bfloat16 format's definition and torch's conversion, the Sec. II-A D_k formula
and the dense Schur complement, a dense residual, finite differences of the loss,
the closed form of Adam's first steps and torch's linear/ReLU layers."""
import numpy as np
import pytest
import torch

from oracle import block, dense, mlp
from paper_2309_06427_gb300 import problems as P


def _probs(shapes, h=0.05):
    return P.custom_problems(shapes, h=h, config=71)


def test_bf16_round_definition_and_torch():
    # ulp of bfloat16 at 1 is 2^-7; ties go to the even significand
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3e-39, 65504.0, 1e38])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == 1 + 2 ** -7 and r[4] == -2.5
    rng = np.random.default_rng(0)
    y = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000), x])
    ref = torch.from_numpy(y.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(y), ref)


@pytest.mark.parametrize("shape", [(5, 3, 2), (7, 14, 7), (3, 28, 14), (4, 6, 0), (0, 4, 2)])
def test_features_rebuild_the_schur_diagonal(shape):
    """Each feature row holds exactly the knot data of S's block row: rebuilding D_k from it by the
    Sec. II-A formula matches the dense C G^-1 C^T, and the D_k^-1 gamma_k slot solves with that block."""
    p = _probs([shape])[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    F = mlp.knot_features(p, S)
    m, u = p.nx, p.nu
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    for k in range(p.N + 1):
        f = F[k]
        A = f[mlp.OFF_A:mlp.OFF_A + 784].reshape(28, 28)
        B = f[mlp.OFF_B:mlp.OFF_B + 392].reshape(28, 14)
        qp, rp = f[mlp.OFF_QP:mlp.OFF_QP + 28], f[mlp.OFF_RP:mlp.OFF_RP + 14]
        q = f[mlp.OFF_Q:mlp.OFF_Q + 28]
        # padding is zero
        assert not A[m:].any() and not A[:, m:].any() and not B[m:].any() and not B[:, u:].any()
        assert not qp[m:].any() and not rp[u:].any() and not q[m:].any()
        Dk = np.diag(1.0 / q[:m].astype(np.float64))
        if k > 0:
            a, b = A[:m, :m], B[:m, :u]
            Dk = Dk + a @ np.diag(1.0 / qp[:m]) @ a.T + b @ np.diag(1.0 / rp[:u]) @ b.T
        blk = Sd[k * m:(k + 1) * m, k * m:(k + 1) * m]
        assert np.allclose(Dk, blk, rtol=1e-12, atol=1e-12)
        g = f[mlp.OFF_G:mlp.OFF_G + m]
        assert np.array_equal(g, p.gamma[k].astype(np.float64))
        assert np.allclose(blk @ f[mlp.OFF_DJ:mlp.OFF_DJ + m], g, rtol=1e-10, atol=1e-12)
        assert f[mlp.OFF_NX] == m / 28 and not f[mlp.OFF_NX + 1:].any()


def test_normalisation_moments():
    probs = _probs([(6, 4), (9, 12), (3, 21)])
    F = np.concatenate([mlp.knot_features(p, block.build_schur(p.A, p.B, p.qd, p.rd)) for p in probs])
    mu, inv = mlp.normalisation(F)
    X = mlp.normalise(F, mu, inv, bf16=False)
    live = inv > 0
    assert np.allclose(X[:, live].mean(0), 0, atol=1e-12) and np.allclose(X[:, live].std(0), 1, atol=1e-9)
    assert not X[:, ~live].any()
    # padding columns and the trailing zero columns are constant
    assert not live[mlp.OFF_NX + 1:].any() and not live[mlp.OFF_A + 27 * 28 + 27]


def test_forward_matches_torch_layers():
    rng = np.random.default_rng(3)
    prm = mlp.unflatten(rng.standard_normal(mlp.N_PARAMS) * 0.05)
    X = rng.standard_normal((37, mlp.D_IN))
    out = mlp.forward(prm, X, bf16=False)
    T = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float64))
    h1 = torch.relu(torch.nn.functional.linear(T(X), T(prm["W1"]), T(prm["b1"])))
    h2 = torch.relu(torch.nn.functional.linear(h1, T(prm["W2"]), T(prm["b2"])))
    y = torch.nn.functional.linear(h2, T(prm["W3"]), T(prm["b3"]))
    assert np.allclose(out["Y"], y.numpy(), rtol=1e-12, atol=1e-12)


def test_loss_is_the_relative_initial_residual():
    probs = _probs([(8, 4), (5, 12)])
    S_list, ls, gs, l0 = [], [], [], []
    rng = np.random.default_rng(5)
    for p in probs:
        S = block.build_schur(p.A, p.B, p.qd, p.rd)
        x = dense.cholesky_solve(dense.schur(p.A, p.B, p.qd, p.rd), p.gamma.astype(np.float64).ravel())
        S_list.append(S); ls.append(x.reshape(p.gamma.shape)); gs.append(p.gamma)
        l0.append(rng.standard_normal(p.gamma.shape) * 0.1)
    # at lambda0 = 0 the loss is ||S lambda*||^2/||gamma||^2 = 1; at lambda0 = lambda* it vanishes
    L0, _ = mlp.loss_and_grad(S_list, [np.zeros_like(x) for x in ls], ls, gs)
    Ls, gstar = mlp.loss_and_grad(S_list, ls, ls, gs)
    assert abs(L0 - 1.0) < 1e-10 and Ls < 1e-20 and max(np.abs(g).max() for g in gstar) < 1e-9
    # equals the dense relative residual of lambda0
    L, _ = mlp.loss_and_grad(S_list, l0, ls, gs)
    ref = np.mean([np.sum((p.gamma.astype(np.float64).ravel() - dense.schur(p.A, p.B, p.qd, p.rd) @ x.ravel()) ** 2)
                   / np.sum(p.gamma.astype(np.float64) ** 2) for p, x in zip(probs, l0)])
    assert abs(L - ref) <= 1e-10 * ref


def test_gradients_match_finite_differences():
    probs = _probs([(6, 4), (4, 6)])
    S_list = [block.build_schur(p.A, p.B, p.qd, p.rd) for p in probs]
    F = np.concatenate([mlp.knot_features(p, S) for p, S in zip(probs, S_list)])
    mu, inv = mlp.normalisation(F)
    X = mlp.normalise(F, mu, inv, bf16=False)
    rng = np.random.default_rng(11)
    prm = mlp.unflatten(rng.standard_normal(mlp.N_PARAMS) * 0.03)
    ls = [rng.standard_normal(p.gamma.shape) for p in probs]
    gs = [p.gamma for p in probs]
    nxs = [p.nx for p in probs]
    rows = [p.n for p in probs]

    def loss(q):
        lam0 = mlp.warm_start(q, X, nxs, rows, bf16=False)
        return mlp.loss_and_grad(S_list, lam0, ls, gs)[0]

    cache = mlp.forward(prm, X, bf16=False)
    lam0, o = [], 0
    for m, r in zip(nxs, rows):
        lam0.append(cache["Y"][o:o + r, :m]); o += r
    _, dl = mlp.loss_and_grad(S_list, lam0, ls, gs)
    grads = mlp.backward(prm, cache, mlp.output_gradient(dl, nxs, bf16=False), bf16=False)
    checked = 0
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = prm[name].ravel()
        idx = rng.choice(flat.size, 6, replace=False)
        if name == "W1":  # include weights on the live gamma and D^-1 gamma columns
            idx = np.concatenate([idx, [5 * mlp.D_IN + mlp.OFF_G, 7 * mlp.D_IN + mlp.OFF_DJ + 1]])
        for i in idx:
            e = 1e-6 * max(1.0, abs(flat[i]))
            qp = {k: v.copy() for k, v in prm.items()}; qp[name].ravel()[i] += e
            qm = {k: v.copy() for k, v in prm.items()}; qm[name].ravel()[i] -= e
            fd = (loss(qp) - loss(qm)) / (2 * e)
            an = grads[name].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (name, i, fd, an)
            checked += 1
    assert checked >= 38


def test_adam_first_steps_closed_form():
    """With bias correction, the first step is -lr g/(|g| + eps); a second step with the same
    gradient again has m_hat = g and v_hat = g^2."""
    rng = np.random.default_rng(2)
    prm = mlp.unflatten(rng.standard_normal(mlp.N_PARAMS))
    g = mlp.unflatten(rng.standard_normal(mlp.N_PARAMS))
    st = {}
    before = mlp.flatten(prm)
    mlp.adam(prm, g, st, lr=1e-3)
    gf = mlp.flatten(g)
    step = -1e-3 * gf / (np.abs(gf) + 1e-8)
    assert np.allclose(mlp.flatten(prm) - before, step, rtol=1e-9, atol=1e-15)
    mid = mlp.flatten(prm)
    mlp.adam(prm, g, st, lr=1e-3)
    assert np.allclose(mlp.flatten(prm) - mid, step, rtol=1e-9, atol=1e-15)


def test_initial_network_predicts_zero_and_training_lowers_the_loss():
    probs = P.make_workload(P.RAGGED_BATCH_4096, count=6)
    S_list = [block.build_schur(p.A, p.B, p.qd, p.rd) for p in probs]
    xs, _, _, _, _, _ = block.solve_batch(probs, "sym", 1e-10)
    F = np.concatenate([mlp.knot_features(p, S) for p, S in zip(probs, S_list)])
    mu, inv = mlp.normalisation(F)
    X = mlp.normalise(F, mu, inv)
    prm = mlp.unflatten(P.mlp_initial_params(0))
    assert not mlp.forward(prm, X)["Y"].any()
    st, losses = {}, []
    for _ in range(40):
        L, _ = mlp.train_step(prm, st, X, S_list, xs, [p.gamma for p in probs], [p.nx for p in probs])
        losses.append(L)
    assert abs(losses[0] - 1.0) < 1e-6 and losses[-1] < 0.9 * losses[0]
