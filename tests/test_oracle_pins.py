"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check ties it to a dense
definition, a closed form worked by hand, a theorem of the paper, the
paper's printed Appendix structure, or brute force.
"""
import os

import numpy as np
import pytest

from oracle import block, dense
from paper_2309_06427_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_n6_block_patterns.txt")

SHAPES = [(0, 1, 1), (0, 3, 2), (1, 1, 1), (1, 2, 1), (2, 3, 2), (3, 2, 2), (4, 4, 2), (5, 3, 1), (7, 2, 1),
          (6, 5, 3)]


def _problems(shapes, h=0.05):
    return P.custom_problems(shapes, h=h, config=77)


@pytest.mark.parametrize("p", _problems(SHAPES), ids=lambda p: f"N{p.N}nx{p.nx}nu{p.nu}")
def test_schur_blocks_equal_dense_definition(p):
    """Sec. II-A: block formulas (theta_k, phi_k, negated) == C G^-1 C^T built densely."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    assert np.allclose(S.dense(), Sd, rtol=0, atol=1e-12 * np.abs(Sd).max())
    assert np.array_equal(S.dense(), S.dense().T)


def test_schur_scalar_closed_form():
    """nx = nu = 1, N = 1 worked by hand: rows [-x0], [a x0 + b u0 - x1].

    S = C G^-1 C^T = [[1/q0, -a/q0], [-a/q0, a^2/q0 + b^2/r0 + 1/q1]].
    """
    a, b, q0, q1, r0 = 0.9, 0.3, 2.0, 5.0, 0.5
    A = np.array([[[a]]]); B = np.array([[[b]]]); qd = np.array([[q0], [q1]]); rd = np.array([[r0]])
    S = block.build_schur(A, B, qd, rd).dense()
    want = np.array([[1 / q0, -a / q0], [-a / q0, a * a / q0 + b * b / r0 + 1 / q1]])
    assert np.allclose(S, want, rtol=1e-15, atol=0)


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _problems(SHAPES[2:]), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_preconditioner_equals_dense_definition(p, kind):
    """Stair-inverse route (Eq. stair_inv) == dense inverses of Psi_l, Psi_r, D (Sec. III, IV)."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, kind)
    Md = dense.preconditioner(S.dense(), p.nx, kind)
    assert np.allclose(M.dense(), Md, rtol=0, atol=1e-10 * np.abs(Md).max())


@pytest.mark.parametrize("p", _problems([(3, 2, 1), (4, 3, 2), (6, 2, 1)]), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_stair_inverse_formula(p):
    """Eq. (stair_inv): Psi^-1 = D^-1 (2D - Psi) D^-1 for both stairs, and S = Psi - P."""
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    D = dense.block_diag_part(Sd, p.nx)
    Di = np.linalg.inv(D)
    Pl_, Pl, Pr_, Pr = dense.stair_splittings(Sd, p.nx)
    for Psi, Pm in ((Pl_, Pl), (Pr_, Pr)):
        assert np.allclose(np.linalg.inv(Psi), Di @ (2 * D - Psi) @ Di, atol=1e-10)
        assert np.allclose(Psi - Pm, Sd, atol=0)
    # Psi_l = Psi_r^T (used in the proof of Thm. 3.5)
    assert np.allclose(Pl_, Pr_.T, atol=0)


@pytest.mark.parametrize("p", _problems([(2, 2, 1), (5, 3, 2), (8, 2, 1)]), ids=lambda p: f"N{p.N}nx{p.nx}")
def test_symmetric_stair_closed_form_and_spd(p):
    """Phi_sym^-1 = 2D^-1 - D^-1 S D^-1 (every off-diagonal block lies in exactly one stair),
    and it is symmetric positive definite."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym").dense()
    Sd = S.dense()
    Di = np.linalg.inv(dense.block_diag_part(Sd, p.nx))
    assert np.allclose(M, 2 * Di - Di @ Sd @ Di, atol=1e-10 * np.abs(M).max())
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def _spectra(p):
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    Sd = S.dense()
    es, ims = dense.spectrum(block.build_precond(S, "sym").dense(), Sd)
    ea, ima = dense.spectrum(block.build_precond(S, "add").dense(), Sd)
    Pl_, Pl, Pr_, Pr = dense.stair_splittings(Sd, p.nx)
    lam_l = np.linalg.eigvals(np.linalg.solve(Pl_, Pl))
    lam_r = np.linalg.eigvals(np.linalg.solve(Pr_, Pr))
    return es, ims, ea, ima, lam_l, lam_r


SPEC = _problems([(2, 2, 1), (3, 2, 1), (4, 3, 2), (5, 2, 1), (6, 3, 1), (9, 2, 1), (10, 1, 1)])


@pytest.mark.parametrize("p", SPEC, ids=lambda p: f"n{p.n}nx{p.nx}")
def test_spectrum_ranges_thm_4_3(p):
    """Thm. 4.3 and Eq. (finalVals): eigenvalues real, sym in (0, 1], add in (0, 9/8]."""
    es, ims, ea, ima, _, _ = _spectra(p)
    assert ims < 1e-8 and ima < 1e-8
    assert es.min() > 0 and es.max() <= 1 + 1e-10
    assert ea.min() > 0 and ea.max() <= 9 / 8 + 1e-10
    # Eq. (max)/(min): the symmetric stair is the better conditioned of the two
    assert es.max() / es.min() < ea.max() / ea.min()


@pytest.mark.parametrize("p", SPEC, ids=lambda p: f"n{p.n}nx{p.nx}")
def test_zero_eigenvalue_counts_and_lemma_3_1(p):
    """Sec. III-A: Psi_l^-1 P_l has m*ceil(n/2) zero and m*floor(n/2) nonzero eigenvalues;
    Lemma 3.1: Psi_l^-1 P_l and Psi_r^-1 P_r share their spectrum."""
    _, _, _, _, lam_l, lam_r = _spectra(p)
    m, n = p.nx, p.n
    scale = max(1.0, np.abs(lam_l).max())
    zero = np.abs(lam_l) < 1e-8 * scale
    assert zero.sum() == m * ((n + 1) // 2)
    assert (~zero).sum() == m * (n // 2)
    a = np.sort_complex(np.round(lam_l, 8)); b = np.sort_complex(np.round(lam_r, 8))
    assert np.allclose(np.sort(np.abs(lam_l)), np.sort(np.abs(lam_r)), atol=1e-8 * scale)
    assert np.allclose(np.sort(lam_l.real), np.sort(lam_r.real), atol=1e-8 * scale)


@pytest.mark.parametrize("p", SPEC, ids=lambda p: f"n{p.n}nx{p.nx}")
def test_thm_4_1_and_4_2_symmetric_spectrum(p):
    """Thm. 4.1/4.2: eig(Phi_sym^-1 S) = {1 (multiplicity m if n odd, else 0)} plus 1 - lambda,
    twice, for every nonzero eigenvalue lambda of Psi_l^-1 P_l."""
    es, _, _, _, lam_l, _ = _spectra(p)
    m, n = p.nx, p.n
    nz = np.sort(lam_l.real[np.abs(lam_l) > 1e-8])
    want = np.sort(np.concatenate([np.ones(m * (n % 2)), 1 - nz, 1 - nz]))
    assert np.allclose(np.sort(es), want, atol=1e-8)
    assert np.sum(np.abs(es - 1) < 1e-8) == m * (n % 2)


@pytest.mark.parametrize("p", SPEC, ids=lambda p: f"n{p.n}nx{p.nx}")
def test_thm_3_3_and_3_4_additive_spectrum(p):
    """Thm. 3.3/3.4: eig(Phi_add^-1 S) = {1 (m if n odd)} plus 1 - (lambda +- sqrt(lambda))/2."""
    _, _, ea, _, lam_l, _ = _spectra(p)
    m, n = p.nx, p.n
    nz = lam_l.real[np.abs(lam_l) > 1e-8]
    assert nz.min() > 0 and nz.max() < 1          # Thm. 4.3 (2): convergent splitting
    s = np.sqrt(nz)
    want = np.sort(np.concatenate([np.ones(m * (n % 2)), 1 - 0.5 * (nz + s), 1 - 0.5 * (nz - s)]))
    assert np.allclose(np.sort(ea), want, atol=1e-8)


def _read_golden():
    pats, name, rows = {}, None, []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("["):
            if name:
                pats[name] = np.array(rows, dtype=int)
            name, rows = line.strip("[]"), []
        else:
            rows.append([int(t) for t in line.split()])
    pats[name] = np.array(rows, dtype=int)
    return pats


def test_appendix_block_patterns_n6():
    """Appendix (Sec. VII), Eq. (lz), (rz), ((l-d)p), (dpl): zero/nonzero block structure at n = 6,
    plus a few printed block values."""
    pats = _read_golden()
    p = _problems([(5, 3, 2)])[0]
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    m = p.nx
    D = dense.block_diag_part(Sd, m)
    Di = np.linalg.inv(D)
    Pl_, Pl, Pr_, Pr = dense.stair_splittings(Sd, m)
    Li, Ri = np.linalg.inv(Pl_), np.linalg.inv(Pr_)
    mats = {
        "Psi_l^-1 P_l": Li @ Pl,
        "Psi_r^-1 P_r": Ri @ Pr,
        "(Psi_l^-1 - D^-1) P_l": (Li - Di) @ Pl,
        "D^-1 P_l": Di @ Pl,
        "(Psi_l^-1 - D^-1) Psi_l": (Li - Di) @ Pl_,
    }
    assert set(mats) == set(pats)
    for name, M in mats.items():
        got = np.array([[int(np.abs(dense.block(M, m, a, b)).max() > 1e-12) for b in range(6)] for a in range(6)])
        assert np.array_equal(got, pats[name]), name
    # printed values (1-based blocks; O_i is S's upper block (i, i+1)); Eq. (lz), (dpl)
    O = lambda i: dense.block(Sd, m, i - 1, i)
    Dinv = lambda i: np.linalg.inv(dense.block(Sd, m, i - 1, i - 1))
    blk = lambda M, a, b: dense.block(M, m, a - 1, b - 1)
    assert np.allclose(blk(mats["Psi_l^-1 P_l"], 1, 2), -Dinv(1) @ O(1), atol=1e-12)
    assert np.allclose(blk(mats["Psi_l^-1 P_l"], 3, 2), -Dinv(3) @ O(2).T, atol=1e-12)
    assert np.allclose(blk(mats["Psi_l^-1 P_l"], 2, 4), Dinv(2) @ O(2) @ Dinv(3) @ O(3), atol=1e-12)
    assert np.allclose(blk(mats["(Psi_l^-1 - D^-1) Psi_l"], 2, 1), -Dinv(2) @ O(1).T, atol=1e-12)
    assert np.allclose(blk(mats["Psi_r^-1 P_r"], 6, 5), -Dinv(6) @ O(5).T, atol=1e-12)


@pytest.mark.parametrize("kind", ["sym", "add", "bj", "jacobi"])
@pytest.mark.parametrize("p", _problems([(0, 3, 2), (1, 2, 1), (6, 3, 2), (20, 2, 1), (12, 5, 3)]),
                         ids=lambda p: f"N{p.N}nx{p.nx}")
def test_pcg_matches_dense_cholesky_and_dense_pcg(p, kind):
    """PCG (Sec. II-B) reaches the unique solution (dense Cholesky) and follows the same
    iterates as an independent dense textbook PCG."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, kind)
    x, it, rr, tr, st = block.pcg(S, M, p.gamma, 1e-12)
    assert st == block.OK and rr <= 1e-12 and tr <= 1e-10
    xd = dense.cholesky_solve(S.dense(), p.gamma)
    assert np.linalg.norm(x.ravel() - xd) <= 1e-8 * np.linalg.norm(xd)
    x2, it2, rr2 = dense.pcg(S.dense(), M.dense(), p.gamma, 1e-8, 10 ** 4)
    x1, it1, rr1, _, _ = block.pcg(S, M, p.gamma, 1e-8)
    assert abs(it1 - it2) <= 1
    assert np.linalg.norm(x1.ravel() - x2) <= 1e-9 * np.linalg.norm(x2) * max(1, it1)


@pytest.mark.parametrize("nx", [1, 2, 4, 6])
def test_special_cases_small_horizons(nx):
    """N = 0: every block preconditioner is exact (1 iteration).  N = 1 (n = 2): Phi_sym^-1 S has
    at most nx distinct eigenvalues; N = 2 (n = 3): at most nx + 1 (Thm. 4.1/4.2).  PCG then ends
    within that many iterations in exact arithmetic (+1 for roundoff)."""
    for N, bound in ((0, 1), (1, nx), (2, nx + 1)):
        p = _problems([(N, nx, max(1, nx // 2))])[0]
        S = block.build_schur(p.A, p.B, p.qd, p.rd)
        for kind in (["sym", "add", "bj"] if N == 0 else ["sym"]):
            _, it, rr, _, st = block.pcg(S, block.build_precond(S, kind), p.gamma, 1e-10)
            assert st == block.OK and it <= bound + 1, (N, kind, it)
            if N == 0:
                assert it == 1


def test_exact_inverse_preconditioner_one_iteration():
    p = _problems([(6, 3, 2)])[0]
    Sd = dense.schur(p.A, p.B, p.qd, p.rd)
    _, it, rr = dense.pcg(Sd, np.linalg.inv(Sd), p.gamma, 1e-10, 100)
    assert it == 1


def test_degenerate_rhs_and_warm_start():
    p = _problems([(5, 3, 2)])[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym")
    x, it, rr, tr, st = block.pcg(S, M, np.zeros_like(p.gamma), 1e-6)
    assert it == 0 and st == block.OK and not x.any()
    xd = dense.cholesky_solve(S.dense(), p.gamma)
    x, it, rr, tr, st = block.pcg(S, M, p.gamma, 1e-6, x0=xd)
    assert it == 0 and st == block.OK


def test_not_positive_definite_is_reported():
    p = _problems([(3, 2, 1)])[0]
    qd = p.qd.copy(); qd[2, 1] = -1.0
    S = block.build_schur(p.A, p.B, qd, p.rd)
    with pytest.raises(np.linalg.LinAlgError):
        block.build_precond(S, "sym")


def test_iteration_ordering_on_pendulum_workload():
    """Sec. V, Fig. 3 (qualitative): symmetric stair needs fewer iterations than the additive
    stair, which needs fewer than block-Jacobi and Jacobi."""
    p = P.make_workload(P.PENDULUM_SINGLE)[0]
    its = {}
    for kind in ("sym", "add", "bj", "jacobi"):
        _, _, _, it, _, _, st = block.solve_problem(p, kind, 1e-8)
        assert st == block.OK
        its[kind] = it
    assert its["sym"] < its["add"] < its["bj"] <= its["jacobi"]


def test_batch_driver_matches_single_problem_path():
    probs = _problems([(3, 2, 1), (0, 3, 2), (9, 4, 2), (5, 1, 1)])
    xs, iters, relres, status, used, dt = block.solve_batch(probs, "sym", 1e-9, nthreads=2)
    assert used >= 1
    for i, p in enumerate(probs):
        _, _, x, it, rr, _, st = block.solve_problem(p, "sym", 1e-9)
        assert status[i] == st and iters[i] == it
        assert np.array_equal(xs[i], x)


def test_pcg_counts_under_reordering():
    """The reorder ensemble: the identity ordering reproduces the dense PCG's count, every reordering solves
    the same system (same solution), a well-conditioned run is fixed to one count, and an ill-conditioned
    scalar-Jacobi run is not (FP64 rounding alone moves its count by more than one)."""
    from paper_2309_06427_gb300 import problems as P
    p = P.make_workload(P.PENDULUM_SINGLE)[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym")
    g = p.gamma.ravel()
    c = dense.pcg_counts_under_reordering(S.dense(), M.dense(), g, 1e-8, 1000, count=8)
    _, it_d, _ = dense.pcg(S.dense(), M.dense(), g, 1e-8, 1000)
    _, it_b, _, _, _ = block.pcg(S, M, p.gamma, 1e-8)
    assert c[0] == c[-1] == it_d == it_b
    perm = np.random.default_rng(3).permutation(g.size)
    ix = np.ix_(perm, perm)
    x_p, _, _ = dense.pcg(S.dense()[ix], M.dense()[ix], g[perm], 1e-12, 1000)
    x, _, _ = dense.pcg(S.dense(), M.dense(), g, 1e-12, 1000)
    assert np.allclose(x_p, x[perm], rtol=1e-9, atol=1e-12)
    shapes = [(0, 1, 1), (0, 5, 3), (1, 2, 1), (2, 3, 2), (7, 4, 2), (20, 2, 1), (33, 12, 6), (64, 14, 7),
              (17, 21, 11), (9, 28, 14), (40, 5, 1)]
    q = P.custom_problems(shapes, h=0.05, config=55)[-1]
    Sq = block.build_schur(q.A, q.B, q.qd, q.rd)
    cj = dense.pcg_counts_under_reordering(Sq.dense(), block.build_precond(Sq, "jacobi").dense(), q.gamma.ravel(),
                                           1e-6, 10000, count=64)
    assert cj[-1] - cj[0] > 1
