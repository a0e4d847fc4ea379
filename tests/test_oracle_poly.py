"""Pins of the oracle's polynomial (Neumann) preconditioner, Eq. polynomial_precon.

Phi_d^-1 = sum_{j<=d} (Psi^-1 P)^j Psi^-1 for the splitting S = Psi - P, with
Psi^-1 one of the assembled preconditioners.  Each pin ties the oracle's
term-by-term application to something built another way: dense matrix
powers of the block-Jacobi splitting, the spectral mapping the series
implies, the exact remainder of a truncated Neumann series, a dense solve.
"""
import numpy as np
import pytest

from oracle import block, dense
from paper_2309_06427_gb300 import problems as P

SHAPES = [(1, 2, 1), (3, 2, 1), (4, 3, 2), (6, 2, 1), (5, 4, 2)]


def _problems(shapes, h=0.05):
    return P.custom_problems(shapes, h=h, config=78)


def _dense_operator(S, M, d):
    """Phi_d^-1 as a dense matrix, one oracle application per unit vector."""
    n = (S.N + 1) * S.nx
    cols = [block.apply_poly(S, M, d, np.eye(n)[:, j]).ravel() for j in range(n)]
    return np.stack(cols, axis=1)


def _setup(p, kind="sym"):
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    return S, block.build_precond(S, kind)


@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_degree_zero_is_the_preconditioner(p):
    S, M = _setup(p)
    assert np.allclose(_dense_operator(S, M, 0), M.dense(), rtol=0, atol=1e-14 * np.abs(M.dense()).max())


@pytest.mark.parametrize("d", [0, 1, 2, 3])
@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_symmetric_stair_series_is_odd_degree_block_jacobi_series(p, d):
    """On Phi_sym (= 2D^-1 - D^-1 S D^-1), degree d equals degree 2d+1 of the block-Jacobi splitting
    S = D - (D - S), here built from dense matrix powers of I - D^-1 S."""
    S, M = _setup(p, "sym")
    Sd = S.dense()
    D = dense.block_diag_part(Sd, p.nx)
    Di = np.linalg.inv(D)
    G = np.eye(len(Sd)) - Di @ Sd
    want = sum(np.linalg.matrix_power(G, j) for j in range(2 * d + 2)) @ Di
    got = _dense_operator(S, M, d)
    assert np.allclose(got, want, rtol=0, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("kind", ["sym", "add", "bj"])
@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_convergent_splitting_and_spectral_mapping(p, kind):
    """rho(Psi^-1 P) = rho(I - Phi^-1 S) < 1 (the paper's validity condition), and the eigenvalues of
    Phi_d^-1 S are 1 - (1 - theta)^(d+1) for the eigenvalues theta of Phi^-1 S; Phi_d^-1 is SPD."""
    S, M = _setup(p, kind)
    Sd, Md = S.dense(), M.dense()
    theta = np.sort(np.linalg.eigvals(Md @ Sd).real)
    assert np.max(np.abs(1 - theta)) < 1
    for d in (1, 2, 3):
        Pd = _dense_operator(S, M, d)
        assert np.allclose(Pd, Pd.T, rtol=0, atol=1e-12 * np.abs(Pd).max())
        assert np.linalg.eigvalsh((Pd + Pd.T) / 2).min() > 0
        mu = np.sort(np.linalg.eigvals(Pd @ Sd).real)
        assert np.allclose(mu, np.sort(1 - (1 - theta) ** (d + 1)), rtol=0, atol=1e-9)


@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_truncation_remainder(p):
    """S^-1 - Phi_d^-1 = (I - Phi^-1 S)^(d+1) S^-1: the tail of the Neumann series."""
    S, M = _setup(p)
    Sd, Md = S.dense(), M.dense()
    Si = np.linalg.inv(Sd)
    G = np.eye(len(Sd)) - Md @ Sd
    for d in (0, 1, 2, 4):
        rem = Si - _dense_operator(S, M, d)
        want = np.linalg.matrix_power(G, d + 1) @ Si
        assert np.allclose(rem, want, rtol=0, atol=1e-9 * np.abs(Si).max())


def test_pcg_with_polynomial_reaches_dense_solution_in_fewer_iterations():
    """Manipulator-like problem (nx = 14, h = 0.01): every degree solves S x = gamma (dense solve), and
    degree 1 takes fewer iterations than degree 0."""
    p = P.make_workload(P.MANIPULATOR_SINGLE, count=1)[0]
    S, M = _setup(p)
    x_ref = np.linalg.solve(S.dense(), p.gamma.astype(np.float64).ravel())
    its = []
    for d in (0, 1, 2, 3):
        x, it, rr, tr, st = block.pcg(S, M, p.gamma, 1e-10, degree=d)
        assert st == block.OK and rr <= 1e-10
        assert np.linalg.norm(x.ravel() - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
        its.append(it)
    assert its[1] < its[0] and its[3] < its[1], its


def test_batch_driver_passes_the_degree():
    probs = _problems([(6, 3, 2), (9, 2, 1), (0, 2, 1)])
    for d in (0, 2):
        xs, iters, _, status, _, _ = block.solve_batch(probs, "sym", 1e-9, degree=d)
        for i, p in enumerate(probs):
            S, M = _setup(p)
            x, it, _, _, st = block.pcg(S, M, p.gamma, 1e-9, degree=d)
            assert status[i] == st == block.OK and iters[i] == it
            assert np.array_equal(xs[i], x)
