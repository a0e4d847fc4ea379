"""Condition number and eigenvalue clustering of Phi^-1 S from the GPU-built
FP32 blocks, against the FP64 oracle's dense eigendecomposition (Sec. IV,
Thm. 4.3; Sec. V, Fig. 1 and Fig. 2), on the manipulator-like and
pendulum-like single-solve workloads."""
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
    from _gpu_helpers import gpu_precond, gpu_schur

KINDS = ("sym", "add", "bj", "jacobi")


def _dense_bt(p, Dd, Eo):
    """Dense symmetric block-tridiagonal matrix from packed GPU blocks (diagonal Dd, sub-diagonal Eo)."""
    n, m = p.n, p.nx
    d = Dd.cpu().numpy()[:n * m * m].reshape(n, m, m).astype(np.float64)
    M = np.zeros((n * m, n * m))
    for k in range(n):
        M[k * m:(k + 1) * m, k * m:(k + 1) * m] = d[k]
    if p.N:
        e = Eo.cpu().numpy()[:p.N * m * m].reshape(p.N, m, m).astype(np.float64)
        for k in range(1, n):
            M[k * m:(k + 1) * m, (k - 1) * m:k * m] = e[k - 1]
            M[(k - 1) * m:k * m, k * m:(k + 1) * m] = e[k - 1].T
    return M


def _spectrum(Minv, S):
    """eig(Phi^-1 S) as the symmetric L^T S L with Phi^-1 = L L^T (real, sorted)."""
    L = np.linalg.cholesky(Minv)
    return np.linalg.eigvalsh(L.T @ S @ L)


def _cases():
    return ([("manipulator", s) for s in range(3)] + [("pendulum", s) for s in range(3)])


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"{c[0]}{c[1]}")
def test_gpu_block_spectra_match_dense_oracle(case):
    w = P.MANIPULATOR_SINGLE if case[0] == "manipulator" else P.PENDULUM_SINGLE
    p = P.make_workload(w, count=1, start=case[1])[0]
    So = block.build_schur(p.A, p.B, p.qd, p.rd)
    _, D, E = gpu_schur(p)
    Sg = _dense_bt(p, D, E)  # the GPU's blocks (measured); the expected spectra use the oracle's own blocks
    kappa = {}
    for kind in KINDS:
        PD, PE, st = gpu_precond(p, D, E, kind)
        assert st == 0
        ev_g = _spectrum(_dense_bt(p, PD, PE), Sg)
        ev_o = np.sort(np.linalg.eigvals(block.build_precond(So, kind).dense() @ So.dense()).real)
        assert np.abs(ev_g - ev_o).max() <= 1e-5, kind
        kg, ko = ev_g[-1] / ev_g[0], ev_o[-1] / ev_o[0]
        assert abs(kg / ko - 1) <= 1e-3, (kind, kg, ko)
        kappa[kind] = kg
        if kind == "sym":   # Thm. 4.3: eigenvalues of Phi_sym^-1 S in (0, 1]
            assert ev_g[0] > 0 and ev_g[-1] <= 1 + 1e-5
        if kind == "add":   # Sec. III: eigenvalues of Phi_add^-1 S in (0, 9/8]
            assert ev_g[0] > 0 and ev_g[-1] <= 9 / 8 + 1e-5
    # Fig. 2 ordering: symmetric stair < additive stair < Jacobi
    assert kappa["sym"] < kappa["add"] < kappa["jacobi"]
