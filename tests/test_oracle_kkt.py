"""Pins of the outer steps of Eq. (schur) in the oracle: gamma formation and the recovery of
delta z, against a dense solve of the whole KKT system and against the paper's block formulas."""
import numpy as np
import pytest

from oracle import block, dense
from paper_2309_06427_gb300 import problems as P


@pytest.mark.parametrize("shape", [(6, 3, 2), (9, 5, 3), (4, 4, 0), (0, 3, 2), (12, 14, 7)])
def test_schur_route_equals_full_kkt_solve(shape):
    p = P.custom_problems([shape], config=73)[0]
    c, q, r = P.qp_vectors(p)
    gam = dense.form_gamma(p.A, p.B, p.qd, p.rd, c, q, r)
    S = dense.schur(p.A, p.B, p.qd, p.rd)
    mu = dense.cholesky_solve(S, gam.ravel()).reshape(gam.shape)
    dx, du = dense.recover_step(p.A, p.B, p.qd, p.rd, q, r, mu)
    kdx, kdu, klam = dense.kkt_solve(p.A, p.B, p.qd, p.rd, c, q, r)
    scale = max(1.0, np.abs(kdx).max())
    assert np.allclose(dx, kdx, atol=1e-9 * scale) and np.allclose(du, kdu, atol=1e-9 * scale)
    assert np.allclose(-mu, klam, atol=1e-9 * max(1.0, np.abs(klam).max()))
    # the step satisfies the constraints and stationarity
    G, C = dense.kkt(p.A, p.B, p.qd, p.rd)
    z = dense._z_vector(dx, du)
    assert np.allclose(C @ z, c.ravel(), atol=1e-9 * scale)
    assert np.allclose(G @ z + C.T @ (-mu.ravel()), dense._z_vector(q, r), atol=1e-8 * scale)


def test_gamma_block_entries():
    """gamma_0 = c_0 + Q_0^-1 q_0 and gamma_{k+1} = c_{k+1} - zeta_k with the paper's
    zeta_k = A_k Q_k^-1 q_k + B_k R_k^-1 r_k - Q_{k+1}^-1 q_{k+1}: the block listing of Sec. II-A
    with the sign of Eq. (schur) (c - C G^-1 g)."""
    p = P.custom_problems([(7, 4, 2)], config=74)[0]
    c, q, r = (a.astype(np.float64) for a in P.qp_vectors(p, seed=3))
    gam = dense.form_gamma(p.A, p.B, p.qd, p.rd, c, q, r)
    A, B, qd, rd = (a.astype(np.float64) for a in (p.A, p.B, p.qd, p.rd))
    assert np.allclose(gam[0], c[0] + q[0] / qd[0], atol=1e-12)
    for k in range(p.N):
        zeta = A[k] @ (q[k] / qd[k]) + B[k] @ (r[k] / rd[k]) - q[k + 1] / qd[k + 1]
        assert np.allclose(gam[k + 1], c[k + 1] - zeta, atol=1e-12)


def test_block_oracle_solution_gives_the_kkt_step():
    """The block oracle's PCG on the formed gamma, then recovery, reaches the dense KKT step."""
    p = P.custom_problems([(20, 6, 3)], config=75)[0]
    c, q, r = P.qp_vectors(p, seed=1)
    gam = dense.form_gamma(p.A, p.B, p.qd, p.rd, c, q, r)
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    mu, it, rr, tr, st = block.pcg(S, block.build_precond(S, "sym"), gam, 1e-12)
    dx, du = dense.recover_step(p.A, p.B, p.qd, p.rd, q, r, mu)
    kdx, kdu, _ = dense.kkt_solve(p.A, p.B, p.qd, p.rd, c, q, r)
    assert st == block.OK
    assert np.linalg.norm(dx - kdx) <= 1e-7 * np.linalg.norm(kdx)
    assert np.linalg.norm(du - kdu) <= 1e-7 * max(np.linalg.norm(kdu), 1e-30)
