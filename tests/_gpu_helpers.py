"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle import block, dense
from paper_2309_06427_gb300 import sspcg

# Parity bar: relative 2-norm error of lambda against the FP64 oracle, and
# iteration counts within one (iters_match).
LAMBDA_RTOL = 1e-5
ITER_TOL = 1
# Problems of at most this many unknowns take the FP64 path in the pipeline
# (same threshold as the library's SSPCG_PRECISION_AUTO).
TINY_UNKNOWNS = 192


def is_tiny(p):
    return p.n * p.nx <= TINY_UNKNOWNS


def reorder_window(p, kind="sym", tol=1e-6, S=None, count=64):
    """(lo, hi): the fewest and most iterations the oracle's dense FP64 textbook PCG takes over ``count``
    symmetric reorderings of the problem's system (S: the oracle's blocks of the system solved; default the
    oracle's FP64 Schur blocks of ``p``).  Oracle only: no value from the CUDA path enters it."""
    if S is None:
        S = block.build_schur(p.A, p.B, p.qd, p.rd)
    M = block.build_precond(S, kind)
    n = S.d.shape[0] * S.d.shape[1]
    c = dense.pcg_counts_under_reordering(S.dense(), M.dense(), p.gamma, tol, 10 * n,
                                          count=count if n <= 3000 else 16)
    return int(c[0]), int(c[-1])


def iters_ok(it_gpu, it_oracle, window=None):
    """Within one of the oracle's count, or of the range ``window`` = (lo, hi)."""
    lo, hi = window if window is not None else (it_oracle, it_oracle)
    return lo - ITER_TOL <= it_gpu <= hi + ITER_TOL


def iters_match(it_gpu, it_oracle, p, kind="sym", tol=1e-6, S=None):
    """Iteration parity: within one of the oracle's count.  Where FP64 arithmetic does not fix the count
    (reordering the oracle's own sums changes it by more than one: ill-conditioned runs, scalar Jacobi), the
    bar is one around the range of the reordered FP64 counts.  That range is only computed when the first
    test fails, and it always contains the oracle's count, so it never narrows the bar."""
    if iters_ok(it_gpu, it_oracle):
        return True
    lo, hi = reorder_window(p, kind, tol, S)
    return iters_ok(it_gpu, it_oracle, (min(lo, it_oracle), max(hi, it_oracle)))


def oracle_blocks32(p):
    """The oracle's FP64 Schur blocks of ``p`` rounded to FP32 on the host: (D [N+1, nx, nx], E [N, nx, nx]
    as float32, and the oracle BlockTridiag of exactly those values).  The block-form GPU calls take these as
    inputs, so that the oracle solves the same FP32 system without reading anything the GPU computed."""
    S = block.build_schur(p.A, p.B, p.qd, p.rd)
    D32 = S.d.astype(np.float32)
    E32 = S.l[1:].astype(np.float32) if p.N > 0 else np.zeros((0, p.nx, p.nx), np.float32)
    d = D32.astype(np.float64)
    l = np.zeros_like(d); u = np.zeros_like(d)
    if p.N > 0:
        l[1:] = E32
        u[:-1] = np.transpose(E32, (0, 2, 1))
    return D32, E32, block.BlockTridiag(d, l, u)


def dev(a, dtype=torch.float32):
    a = np.ascontiguousarray(a)
    if a.size == 0:
        a = np.zeros(4, dtype=a.dtype)
    return torch.from_numpy(a).to(dtype).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel(); b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_schur(p):
    n, m = p.n, p.nx
    A, B, qd, rd = dev(p.A), dev(p.B), dev(p.qd), dev(p.rd)
    D = torch.zeros(max(n * m * m, 4), device="cuda")
    E = torch.zeros(max(p.N * m * m, 4), device="cuda")
    sspcg.sspcg_build_schur(p.N, m, p.nu, A, B, qd, rd, D, E)
    return (A, B, qd, rd), D, E


def gpu_precond(p, D, E, kind):
    n, m = p.n, p.nx
    PD = torch.zeros(max(n * m * m, 4), device="cuda")
    PE = torch.zeros(max(p.N * m * m, 4), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_precond(p.N, m, kind, D, E, PD, PE, st)
    return PD, PE, int(st.item())


def gpu_solve_qp(p, kind="sym", tol=1e-6, lam0=None, **kw):
    """Whole single-problem path on the GPU: returns (lambda, iters, relres, status)."""
    (A, B, qd, rd), D, E = gpu_schur(p)
    PD, PE, pst = gpu_precond(p, D, E, kind)
    g = dev(p.gamma)
    lam = dev(lam0) if lam0 is not None else torch.zeros_like(g)
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = sspcg.options(tol=tol, warm_start=0 if lam0 is None else kw.pop("warm", 1), **kw)
    sspcg.sspcg_solve_qp(p.N, p.nx, p.nu, A, B, qd, rd, PD, PE, g, lam, opts, it, rr, st)
    torch.cuda.synchronize()
    return lam.cpu().numpy()[:p.gamma.size].reshape(p.gamma.shape), int(it.item()), float(rr.item()), int(st.item())


def gpu_solve_qp_f64(p, kind="sym", tol=1e-6, **kw):
    """Whole single-problem path on the GPU in FP64: returns (lambda, iters, relres, status)."""
    n, m = p.n, p.nx
    A, B, qd, rd = dev(p.A), dev(p.B), dev(p.qd), dev(p.rd)
    D = torch.zeros(max(n * m * m, 2), dtype=torch.float64, device="cuda")
    E = torch.zeros(max(p.N * m * m, 2), dtype=torch.float64, device="cuda")
    PD, PE = torch.zeros_like(D), torch.zeros_like(E)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sspcg.sspcg_build_schur_f64(p.N, m, p.nu, A, B, qd, rd, D, E)
    sspcg.sspcg_build_precond_f64(p.N, m, kind, D, E, PD, PE, st)
    g = dev(p.gamma)
    lam = torch.zeros(max(n * m, 2), dtype=torch.float64, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    sspcg.sspcg_solve_qp_f64(p.N, m, p.nu, A, B, qd, rd, PD, PE, g, lam, sspcg.options(tol=tol, **kw), it, rr, st)
    torch.cuda.synchronize()
    return lam.cpu().numpy()[:p.gamma.size].reshape(p.gamma.shape), int(it.item()), float(rr.item()), int(st.item())


def gpu_solve_auto(p, kind="sym", tol=1e-6, **kw):
    """The precision the batched pipeline uses for this problem (FP64 when tiny)."""
    return gpu_solve_qp_f64(p, kind, tol, **kw) if is_tiny(p) else gpu_solve_qp(p, kind, tol, **kw)
