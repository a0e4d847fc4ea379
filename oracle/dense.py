"""Dense FP64 definitions (numpy/scipy) for tiny and medium problems.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``kkt``: the QP of Sec. II-A as dense matrices.  Variables are ordered
  z = (x_0, u_0, x_1, u_1, ..., x_{N-1}, u_{N-1}, x_N); G is the cost Hessian
  blockdiag(Q_0, R_0, ..., Q_N); the constraint Jacobian C has one block row
  for the initial state (-x_0 + x_s = 0) and one per knot
  (A_k x_k + B_k u_k - x_{k+1} = 0).
* ``schur``: S = C G^-1 C^T, the positive definite form of Eq. (schur)
  (the footnote of Sec. II-A negates the paper's -C G^-1 C^T).  ``kkt_full``,
  ``schur_full``: the same with full SPD cost blocks Q_k, R_k.
* ``stair_splittings``: Psi_l, P_l, Psi_r, P_r by the block patterns of
  Eq. (stair) (Psi_l keeps the off-diagonal blocks of the even 1-based block
  rows, Psi_r of the odd rows; S = Psi - P).
* ``preconditioner``: Phi^-1 by dense LAPACK inverses of those definitions:
  Sec. IV (symmetric stair), Sec. III (additive stair), Eq. (jacobi).
* ``cholesky_solve``: the exact solution of S x = gamma.
* ``pcg``: textbook PCG on dense matrices (Saad, Alg. 9.1).
* ``pcg_counts_under_reordering``: its iteration counts over symmetric
  reorderings of one system (how far FP64 rounding fixes the count).
* ``form_gamma``, ``recover_step``: the two outer steps of Eq. (schur), written
  densely: gamma = c - C G^-1 g and delta z = G^-1 (g - C^T lambda*), with the
  paper's lambda* = -mu (mu solves C G^-1 C^T mu = gamma).  ``kkt_solve``: the
  same QP step by one dense solve of the whole KKT system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def kkt(A, B, qd, rd):
    """Dense (G, C) of the trajectory QP for diagonal Q_k = diag(qd[k]), R_k = diag(rd[k])."""
    qd, rd = np.asarray(qd, dtype=np.float64), np.asarray(rd, dtype=np.float64)
    Q = np.stack([np.diag(q) for q in qd])
    R = np.stack([np.diag(r) for r in rd]) if len(rd) else np.zeros((0, 0, 0))
    return kkt_full(A, B, Q, R)


def kkt_full(A, B, Q, R):
    """Dense (G, C) of the trajectory QP with full SPD cost blocks Q [N+1][nx][nx], R [N][nu][nu]:
    G = blockdiag(Q_0, R_0, ..., R_{N-1}, Q_N)."""
    A, B, Q = (np.asarray(a, dtype=np.float64) for a in (A, B, Q))
    N, nx = Q.shape[0] - 1, Q.shape[1]
    nu = B.shape[2] if N > 0 else 0
    R = np.asarray(R, dtype=np.float64).reshape(N, nu, nu)
    nz = (N + 1) * nx + N * nu
    xo = lambda k: k * (nx + nu)           # column offset of x_k
    uo = lambda k: k * (nx + nu) + nx      # column offset of u_k
    G = np.zeros((nz, nz))
    for k in range(N + 1):
        G[xo(k):xo(k) + nx, xo(k):xo(k) + nx] = Q[k]
        if k < N:
            G[uo(k):uo(k) + nu, uo(k):uo(k) + nu] = R[k]
    C = np.zeros(((N + 1) * nx, nz))
    C[0:nx, xo(0):xo(0) + nx] = -np.eye(nx)
    for k in range(N):
        rows = slice((k + 1) * nx, (k + 2) * nx)
        C[rows, xo(k):xo(k) + nx] = A[k]
        C[rows, uo(k):uo(k) + nu] = B[k]
        C[rows, xo(k + 1):xo(k + 1) + nx] = -np.eye(nx)
    return G, C


def schur(A, B, qd, rd) -> np.ndarray:
    G, C = kkt(A, B, qd, rd)
    return C @ np.linalg.solve(G, C.T)


def schur_full(A, B, Q, R) -> np.ndarray:
    """S = C G^-1 C^T with full SPD cost blocks."""
    G, C = kkt_full(A, B, Q, R)
    return C @ np.linalg.solve(G, C.T)


def block(M, nx, a, b):
    return M[a * nx:(a + 1) * nx, b * nx:(b + 1) * nx]


def block_diag_part(S, nx) -> np.ndarray:
    n = S.shape[0] // nx
    D = np.zeros_like(S)
    for k in range(n):
        D[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx] = block(S, nx, k, k)
    return D


def stair_splittings(S, nx):
    """(Psi_l, P_l, Psi_r, P_r) with S = Psi_l - P_l = Psi_r - P_r (Eq. stair)."""
    n = S.shape[0] // nx
    D = block_diag_part(S, nx)
    Psi_l, Psi_r = D.copy(), D.copy()
    for k in range(n):              # 0-based k is 1-based row k+1
        target = Psi_l if (k + 1) % 2 == 0 else Psi_r
        for j in (k - 1, k + 1):
            if 0 <= j < n:
                target[k * nx:(k + 1) * nx, j * nx:(j + 1) * nx] = block(S, nx, k, j)
    return Psi_l, Psi_l - S, Psi_r, Psi_r - S


def preconditioner(S, nx, kind="sym") -> np.ndarray:
    """Phi^-1 from its definition by dense inverses."""
    if kind == "jacobi":
        return np.diag(1.0 / np.diag(S))
    D = block_diag_part(S, nx)
    Dinv = np.linalg.inv(D)
    if kind == "bj":
        return Dinv
    Psi_l, _, Psi_r, _ = stair_splittings(S, nx)
    Li, Ri = np.linalg.inv(Psi_l), np.linalg.inv(Psi_r)
    if kind == "sym":
        return Li + Ri - Dinv
    if kind == "add":
        return 0.5 * (Li + Ri)
    raise ValueError(kind)


def cholesky_solve(S, gamma) -> np.ndarray:
    c = scipy.linalg.cho_factor(S, lower=True)
    return scipy.linalg.cho_solve(c, np.asarray(gamma, dtype=np.float64).ravel())


def pcg(S, Minv, gamma, tol, max_iter, x0=None):
    """Textbook PCG on dense matrices.  Returns (x, iters, relres)."""
    g = np.asarray(gamma, dtype=np.float64).ravel()
    gn = np.linalg.norm(g)
    if gn == 0.0:
        return np.zeros_like(g), 0, 0.0
    x = np.zeros_like(g) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    r = g - S @ x
    z = Minv @ r
    p = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > tol * gn and it < max_iter:
        w = S @ p
        alpha = rz / (p @ w)
        x += alpha * p
        r -= alpha * w
        z = Minv @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, np.linalg.norm(r) / gn


def pcg_counts_under_reordering(S, Minv, gamma, tol, max_iter, count=64, seed=0):
    """Iteration counts of the textbook PCG (``pcg``) on ``count`` symmetric reorderings of the same system:
    P S P^T y = P gamma with the preconditioner P Phi^-1 P^T, P a seeded random permutation (the first one
    the identity).  In exact arithmetic every reordering takes the same iterations, so the spread of the
    counts is what FP64 rounding alone (the order of its sums) leaves undetermined.  Returns a sorted array."""
    g = np.asarray(gamma, dtype=np.float64).ravel()
    rng = np.random.default_rng(seed)
    counts = []
    for t in range(count):
        perm = np.arange(g.size) if t == 0 else rng.permutation(g.size)
        ix = np.ix_(perm, perm)
        counts.append(pcg(S[ix], Minv[ix], g[perm], tol, max_iter)[1])
    return np.sort(np.array(counts))


def spectrum(Minv, S) -> np.ndarray:
    """Eigenvalues of Phi^-1 S (real by similarity, footnote of Sec. III), ascending."""
    ev = np.linalg.eigvals(Minv @ S)
    return np.sort(ev.real), np.max(np.abs(ev.imag))


def condition_number(Minv, S) -> float:
    ev, _ = spectrum(Minv, S)
    return ev[-1] / ev[0]


def _z_vector(q, r):
    """Stack state and input vectors in the variable order of ``kkt`` (x_0, u_0, ..., x_N)."""
    q, r = np.asarray(q, dtype=np.float64), np.asarray(r, dtype=np.float64)
    N = q.shape[0] - 1
    parts = []
    for k in range(N + 1):
        parts.append(q[k])
        if k < N:
            parts.append(r[k])
    return np.concatenate(parts) if parts else np.zeros(0)


def _split_z(z, N, nx, nu):
    dx = np.zeros((N + 1, nx)); du = np.zeros((N, nu))
    o = 0
    for k in range(N + 1):
        dx[k] = z[o:o + nx]; o += nx
        if k < N:
            du[k] = z[o:o + nu]; o += nu
    return dx, du


def form_gamma(A, B, qd, rd, c, q, r) -> np.ndarray:
    """gamma = c - C G^-1 g (Eq. schur), g = (q_0, r_0, ..., q_N); returned as [N+1, nx]."""
    G, C = kkt(A, B, qd, rd)
    g = _z_vector(q, r)
    c = np.asarray(c, dtype=np.float64)
    return (c.ravel() - C @ np.linalg.solve(G, g)).reshape(c.shape)


def recover_step(A, B, qd, rd, q, r, mu):
    """delta z = G^-1 (g - C^T lambda*) with lambda* = -mu (Eq. schur): (dx [N+1, nx], du [N, nu])."""
    G, C = kkt(A, B, qd, rd)
    g = _z_vector(q, r)
    lam = -np.asarray(mu, dtype=np.float64).ravel()
    z = np.linalg.solve(G, g - C.T @ lam)
    qd = np.asarray(qd)
    N, nx = qd.shape[0] - 1, qd.shape[1]
    nu = np.asarray(r).shape[1] if N > 0 else 0
    return _split_z(z, N, nx, nu)


def kkt_solve(A, B, qd, rd, c, q, r):
    """The QP step from one dense solve of [[G, C^T], [C, 0]] [z; lambda] = [g; c] (the KKT system of
    minimising z^T G z / 2 - g^T z subject to C z = c): (dx, du, lambda [N+1, nx])."""
    G, C = kkt(A, B, qd, rd)
    g = _z_vector(q, r)
    nz, nc = G.shape[0], C.shape[0]
    K = np.block([[G, C.T], [C, np.zeros((nc, nc))]])
    sol = np.linalg.solve(K, np.concatenate([g, np.asarray(c, dtype=np.float64).ravel()]))
    qd = np.asarray(qd)
    N, nx = qd.shape[0] - 1, qd.shape[1]
    nu = np.asarray(r).shape[1] if N > 0 else 0
    dx, du = _split_z(sol[:nz], N, nx, nu)
    return dx, du, sol[nz:].reshape(N + 1, nx)

