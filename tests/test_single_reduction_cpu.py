"""The single-reduction (Chronopoulos-Gear) recurrences the GPU kernel's cg_variant = 1 uses, written
here in FP64 numpy: s = S p kept by recurrence, and alpha from (r.u, S u.u) alone through
p.S p = S u.u - beta (r.u) / alpha_old.  In exact arithmetic they give the textbook PCG iterates, so on
small problems they must reproduce the oracle's textbook PCG (iterates and iteration counts)."""
import numpy as np
import pytest

from oracle import block
from paper_2309_06427_gb300 import problems as P


def single_reduction_pcg(S, M, g, tol, max_iter):
    x = np.zeros_like(g)
    r = g.copy()
    u = M @ r
    w = S @ u
    ru, dl, rr = r @ u, w @ u, r @ r
    gg = g @ g
    alpha, beta, it = ru / dl, 0.0, 0
    p = s = None
    while rr > tol * tol * gg and it < max_iter:
        p = u if it == 0 else u + beta * p
        s = w if it == 0 else w + beta * s
        x = x + alpha * p
        r = r - alpha * s
        u = M @ r
        w = S @ u
        ru_old = ru
        ru, dl, rr = r @ u, w @ u, r @ r
        it += 1
        beta = ru / ru_old
        alpha = ru / (dl - beta * ru / alpha)
    return x, it


@pytest.mark.parametrize("p", P.custom_problems([(6, 3, 2), (12, 4, 2), (20, 2, 1), (9, 5, 3)], config=89),
                         ids=lambda p: f"N{p.N}nx{p.nx}")
@pytest.mark.parametrize("kind", ["sym", "add", "bj"])
def test_single_reduction_recurrences_give_the_textbook_iterates(p, kind):
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, kind)
    g = p.gamma.astype(np.float64).ravel()
    x_o, it_o, _, _, st = block.pcg(S, M, p.gamma, 1e-9)
    x, it = single_reduction_pcg(S.dense(), M.dense(), g, 1e-9, 10 * g.size)
    assert st == block.OK and abs(it - it_o) <= 1
    assert np.linalg.norm(x - x_o.ravel()) <= 1e-7 * np.linalg.norm(x_o)
    # the same iterate after a fixed number of steps, before convergence
    k = max(1, it_o // 2)
    x_k, _, _, _, _ = block.pcg(S, M, p.gamma, 1e-9, max_iter=k)
    xs, its = single_reduction_pcg(S.dense(), M.dense(), g, 1e-9, k)
    assert its == k and np.linalg.norm(xs - x_k.ravel()) <= 1e-8 * np.linalg.norm(x_k)


def test_a_wrong_alpha_recurrence_is_caught():
    """Dropping the beta term of the p.S p identity gives different iterates: the pin above would fail."""
    p = P.custom_problems([(12, 4, 2)], config=89)[0]
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, "sym")
    Sd, Md, g = S.dense(), M.dense(), p.gamma.astype(np.float64).ravel()
    x_k, _, _, _, _ = block.pcg(S, M, p.gamma, 1e-12, max_iter=5)
    # planted mistake: alpha = (r.u) / (S u.u)
    x = np.zeros_like(g); r = g.copy(); u = Md @ r; w = Sd @ u
    ru, dl = r @ u, w @ u
    alpha, beta, pp, ss = ru / dl, 0.0, None, None
    for it in range(5):
        pp = u if it == 0 else u + beta * pp
        ss = w if it == 0 else w + beta * ss
        x = x + alpha * pp
        r = r - alpha * ss
        u = Md @ r; w = Sd @ u
        ru_old = ru
        ru, dl = r @ u, w @ u
        beta = ru / ru_old
        alpha = ru / dl
    assert np.linalg.norm(x - x_k.ravel()) > 1e-4 * np.linalg.norm(x_k)
