"""Pins of the oracle's Schur build with full SPD cost blocks Q_k, R_k (Sec. II-A,
where the block formulas carry Q_k^-1 and R_k^-1 as matrices).

Each check ties oracle_build_schur_full to the dense definition C G^-1 C^T with
a block-diagonal G, to the diagonal-cost routine on diagonal inputs, or to a
property that holds for every SPD block-tridiagonal S.
"""
import numpy as np
import pytest

from oracle import block, dense
from paper_2309_06427_gb300 import problems as P

SHAPES = [(0, 3, 2), (1, 1, 1), (1, 2, 1), (3, 2, 2), (4, 3, 2), (5, 4, 1), (6, 5, 3), (3, 3, 0)]


def _problems(shapes, h=0.05):
    return P.custom_problems(shapes, h=h, config=81)


@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_full_schur_equals_dense_definition(p):
    Q, R = P.full_cost(p)
    S = block.build_schur_full(p.A, p.B, Q, R)
    Sd = dense.schur_full(p.A, p.B, Q, R)
    assert np.allclose(S.dense(), Sd, rtol=0, atol=1e-12 * np.abs(Sd).max())
    # inverses by Cholesky solves are symmetric to rounding only
    assert np.allclose(S.dense(), S.dense().T, rtol=0, atol=1e-14 * np.abs(Sd).max())
    assert np.linalg.eigvalsh(Sd).min() > 0


@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_diagonal_cost_reduces_to_the_diagonal_routine(p):
    Q = np.stack([np.diag(q) for q in p.qd.astype(np.float64)])
    R = np.stack([np.diag(r) for r in p.rd.astype(np.float64)]) if p.N else np.zeros((0, p.nu, p.nu))
    Sf = block.build_schur_full(p.A, p.B, Q, R).dense()
    Sd = block.build_schur(p.A, p.B, p.qd, p.rd).dense()
    assert np.allclose(Sf, Sd, rtol=0, atol=1e-13 * np.abs(Sd).max())


def test_scalar_closed_form_with_coupled_cost():
    """nx = 1, nu = 2, N = 1 by hand: S = [[1/q0, -a/q0], [-a/q0, a^2/q0 + b^T R^-1 b + 1/q1]]."""
    a, q0, q1 = 0.9, 2.0, 5.0
    b = np.array([0.3, -0.2])
    Rm = np.array([[0.5, 0.1], [0.1, 0.8]])
    A = np.array([[[a]]]); B = b.reshape(1, 1, 2); Q = np.array([[[q0]], [[q1]]]); R = Rm.reshape(1, 2, 2)
    S = block.build_schur_full(A, B, Q, R).dense()
    want = np.array([[1 / q0, -a / q0], [-a / q0, a * a / q0 + b @ np.linalg.solve(Rm, b) + 1 / q1]])
    assert np.allclose(S, want, rtol=1e-14, atol=0)


def test_generator_gives_symmetric_positive_definite_blocks():
    for p in _problems([(4, 6, 3), (2, 28, 14), (0, 5, 3)]):
        Q, R = P.full_cost(p)
        assert Q.shape == (p.N + 1, p.nx, p.nx) and R.shape == (p.N, p.nu, p.nu)
        assert np.array_equal(Q, np.swapaxes(Q, 1, 2)) and np.array_equal(R, np.swapaxes(R, 1, 2))
        for k in range(p.N + 1):
            assert np.linalg.eigvalsh(Q[k].astype(np.float64) - np.diag(p.qd[k])).min() > -1e-5
        assert all(np.linalg.eigvalsh(R[k]).min() > 0 for k in range(p.N))
        Q2, R2 = P.full_cost(p)
        assert np.array_equal(Q, Q2) and np.array_equal(R, R2)


def test_indefinite_cost_block_is_reported():
    p = _problems([(3, 3, 2)])[0]
    Q, R = P.full_cost(p)
    Q = Q.astype(np.float64)
    Q[2] = -Q[2]
    with pytest.raises(np.linalg.LinAlgError):
        block.build_schur_full(p.A, p.B, Q, R)
    Q, R = P.full_cost(p)
    R = R.astype(np.float64)
    R[1, 0, 0] = -1.0
    with pytest.raises(np.linalg.LinAlgError):
        block.build_schur_full(p.A, p.B, Q, R)


@pytest.mark.parametrize("p", _problems([(6, 3, 2), (9, 4, 2)]), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_stair_theory_and_pcg_hold_with_full_cost(p):
    """The stair results need only an SPD block-tridiagonal S: eig(Phi_sym^-1 S) in (0, 1] (Thm. 4.3),
    and PCG with Phi_sym reaches the dense solution."""
    Q, R = P.full_cost(p)
    S = block.build_schur_full(p.A, p.B, Q, R)
    M = block.build_precond(S, "sym")
    ev = np.linalg.eigvals(M.dense() @ S.dense()).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10
    x, it, rr, tr, st = block.pcg(S, M, p.gamma, 1e-10)
    x_ref = np.linalg.solve(S.dense(), p.gamma.astype(np.float64).ravel())
    assert st == block.OK and np.linalg.norm(x.ravel() - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
