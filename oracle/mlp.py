"""FP64 oracle of the learned warm start: knot features, the 3-layer ReLU
network, its loss, gradients and the Adam update.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; what is computed here is this project's
definition of the warm start, written out plainly so that the CUDA kernels can
be checked against it:

* Knot features (one row per block row k of S).  Block row k of the Schur
  complement is built from the knot data (A_{k-1}, B_{k-1}, Q_{k-1}, R_{k-1},
  Q_k) by the D_k formula of Sec. II-A; the row carries those data, zero padded
  to nx = 28, nu = 14, plus gamma_k, the block-diagonal solve D_k^-1 gamma_k and
  nx/28.  Layout of the D_IN = 1344 columns:

      [0, 784)      A_{k-1}  as [28][28] row-major   (zero for k = 0)
      [784, 1176)   B_{k-1}  as [28][14] row-major   (zero for k = 0)
      [1176, 1204)  diag Q_{k-1}                     (zero for k = 0)
      [1204, 1218)  diag R_{k-1}                     (zero for k = 0)
      [1218, 1246)  diag Q_k
      [1246, 1274)  gamma_k
      [1274, 1302)  D_k^-1 gamma_k
      1302          nx / 28
      [1303, 1344)  zero

* Normalisation: column mean mu and 1/sigma over the training rows (population
  standard deviation); a column whose sigma is at most 1e-6 of its RMS is
  constant and gets 1/sigma = 0.
* Network: H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3
  with W1 [256][1344], W2 [256][256], W3 [32][256]; lambda0_k = Y[k, :nx].
  The CUDA path stores X, H1, H2, the weights used by the products and the
  output gradient in bfloat16; ``bf16=True`` rounds at the same points
  (round to nearest even), everything else is FP64.
* Loss of one problem: the squared S^2-norm of the warm start's error,
  ||S (lambda0 - lambda*)||^2 / ||gamma||^2, averaged over the problems of a
  minibatch.  With lambda* the plain method's solution (S lambda* = gamma up to
  its tolerance) this is the squared relative initial residual that the PCG
  exit test (relative to ||gamma||) measures.  Its gradient with respect to
  lambda0 is 2 S S (lambda0 - lambda*) / ||gamma||^2 / P.
* Adam (Kingma & Ba, 2015, Algorithm 1) on FP32 master weights.
"""
from __future__ import annotations

import numpy as np

NXM, NUM = 28, 14
D_IN, HID, OUT = 1344, 256, 32
OFF_A, OFF_B, OFF_QP, OFF_RP, OFF_Q, OFF_G, OFF_DJ, OFF_NX = 0, 784, 1176, 1204, 1218, 1246, 1274, 1302
SHAPES = (("W1", (HID, D_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)),
          ("b3", (OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of
    an IEEE binary32 value: round the binary32 value at bit 16."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(np.shape(x))


def knot_features(p, S) -> np.ndarray:
    """Raw feature rows [N+1, D_IN] of problem ``p`` (FP64); ``S`` is its FP64 block Schur
    complement (``oracle.block.build_schur``), whose diagonal blocks give D_k^-1 gamma_k."""
    n, m, u = p.N + 1, p.nx, p.nu
    F = np.zeros((n, D_IN))
    g = np.asarray(p.gamma, dtype=np.float64)
    for k in range(n):
        if k > 0:
            a = np.zeros((NXM, NXM)); a[:m, :m] = p.A[k - 1]
            F[k, OFF_A:OFF_A + NXM * NXM] = a.ravel()
            if u > 0:
                b = np.zeros((NXM, NUM)); b[:m, :u] = p.B[k - 1]
                F[k, OFF_B:OFF_B + NXM * NUM] = b.ravel()
                F[k, OFF_RP:OFF_RP + u] = p.rd[k - 1]
            F[k, OFF_QP:OFF_QP + m] = p.qd[k - 1]
        F[k, OFF_Q:OFF_Q + m] = p.qd[k]
        F[k, OFF_G:OFF_G + m] = g[k]
        F[k, OFF_DJ:OFF_DJ + m] = np.linalg.solve(S.d[k], g[k])
        F[k, OFF_NX] = m / NXM
    return F


def normalisation(F: np.ndarray):
    """(mu, inv_sigma) of the rows of F."""
    F = np.asarray(F, dtype=np.float64)
    mu = F.mean(axis=0)
    ms = (F * F).mean(axis=0)
    var = np.maximum(ms - mu * mu, 0.0)
    sig = np.sqrt(var)
    const = sig <= 1e-6 * np.sqrt(ms)
    inv = np.where(const, 0.0, 1.0 / np.where(const, 1.0, sig))
    return mu, inv


def normalise(F, mu, inv_sigma, bf16=True) -> np.ndarray:
    X = (np.asarray(F, dtype=np.float64) - mu) * inv_sigma
    return bf16_round(X) if bf16 else X


def unflatten(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64).ravel()
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        size = int(np.prod(shp))
        out[name] = flat[o:o + size].reshape(shp).copy()
        o += size
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(params: dict, X, bf16=True) -> dict:
    """The three layers on normalised features X [rows, D_IN]."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = rnd(params["W1"]), rnd(params["W2"]), rnd(params["W3"])
    Z1 = X @ W1.T + params["b1"]
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + params["b2"]
    H2 = rnd(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + params["b3"]
    return {"X": X, "H1": H1, "H2": H2, "Y": Y}


def bt_apply(S, x) -> np.ndarray:
    """y = S x for a block tridiagonal S (d, l, u blocks) and x [N+1, nx]."""
    y = np.einsum("kij,kj->ki", S.d, x)
    if S.d.shape[0] > 1:
        y[1:] += np.einsum("kij,kj->ki", S.l[1:], x[:-1])
        y[:-1] += np.einsum("kij,kj->ki", S.u[:-1], x[1:])
    return y


def loss_and_grad(S_list, lam0_list, lamstar_list, gamma_list):
    """Minibatch loss (mean over problems of ||S(lambda0 - lambda*)||^2 / ||gamma||^2) and its
    gradient with respect to every lambda0."""
    P = len(S_list)
    total, grads = 0.0, []
    for S, l0, ls, g in zip(S_list, lam0_list, lamstar_list, gamma_list):
        gg = float(np.sum(np.asarray(g, dtype=np.float64) ** 2))
        gg = gg if gg > 0 else 1.0
        u = bt_apply(S, np.asarray(l0, dtype=np.float64) - np.asarray(ls, dtype=np.float64))
        total += float(np.sum(u * u)) / gg
        grads.append(2.0 * bt_apply(S, u) / gg / P)
    return total / P, grads


def output_gradient(dlam_list, nx_list, bf16=True) -> np.ndarray:
    """dL/dY [rows, OUT]: the lambda0 gradients in the first nx columns, zero elsewhere."""
    rows = []
    for dl, m in zip(dlam_list, nx_list):
        d = np.zeros((dl.shape[0], OUT)); d[:, :m] = dl
        rows.append(d)
    dY = np.concatenate(rows) if rows else np.zeros((0, OUT))
    return bf16_round(dY) if bf16 else dY


def backward(params: dict, cache: dict, dY, bf16=True) -> dict:
    """Gradients of the three layers given dL/dY (chain rule through the ReLUs)."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W2, W3 = rnd(params["W2"]), rnd(params["W3"])
    X, H1, H2 = cache["X"], cache["H1"], cache["H2"]
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dH2 = rnd((dY @ W3) * (H2 > 0))
    g["W2"] = dH2.T @ H1
    g["b2"] = dH2.sum(axis=0)
    dH1 = rnd((dH2 @ W2) * (H1 > 0))
    g["W1"] = dH1.T @ X
    g["b1"] = dH1.sum(axis=0)
    return g


def adam(params: dict, grads: dict, state: dict, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam step in place (Kingma & Ba, Algorithm 1); ``state`` holds t, m, v."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for name, _ in SHAPES:
        m = state.setdefault("m_" + name, np.zeros_like(params[name]))
        v = state.setdefault("v_" + name, np.zeros_like(params[name]))
        gr = grads[name]
        m[...] = beta1 * m + (1.0 - beta1) * gr
        v[...] = beta2 * v + (1.0 - beta2) * gr * gr
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[name] = params[name] - lr * mhat / (np.sqrt(vhat) + eps)


def warm_start(params: dict, X, nx_list, rows_list, bf16=True):
    """lambda0 of each problem (rows of X in problem order)."""
    Y = forward(params, X, bf16)["Y"]
    out, o = [], 0
    for m, r in zip(nx_list, rows_list):
        out.append(Y[o:o + r, :m].copy())
        o += r
    return out


def train_step(params: dict, state: dict, X, S_list, lamstar_list, gamma_list, nx_list, lr=1e-3, bf16=True):
    """Forward, loss, backward and Adam on one minibatch of whole problems; returns (loss, grads)."""
    rows = [ls.shape[0] for ls in lamstar_list]
    cache = forward(params, X, bf16)
    lam0, o = [], 0
    for m, r in zip(nx_list, rows):
        lam0.append(cache["Y"][o:o + r, :m])
        o += r
    loss, dl = loss_and_grad(S_list, lam0, lamstar_list, gamma_list)
    dY = output_gradient(dl, nx_list, bf16)
    grads = backward(params, cache, dY, bf16)
    adam(params, grads, state, lr)
    return loss, grads
