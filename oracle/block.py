"""ctypes front end of the FP64 block oracle (``sspcg_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build()`` compiles
the C file with gcc into ``oracle/_lib/liboracle.so``; the functions below
take and return float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sspcg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

SYM_STAIR, ADD_STAIR, BLOCK_JACOBI, JACOBI = 0, 1, 2, 3
KINDS = {"sym": SYM_STAIR, "add": ADD_STAIR, "bj": BLOCK_JACOBI, "jacobi": JACOBI}
OK, MAXITER, BREAKDOWN, NOT_SPD, NONFINITE, BADARG = 0, 1, 2, 3, 4, 5

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3, ISO C11, OpenMP when the compiler has it).

    No -march=native: the same source builds on x86 and Arm hosts and must give the same results on both;
    in ISO C mode gcc neither contracts a*b+c into FMAs nor reassociates sums, so -O3 changes no result."""
    os.makedirs(_LIBDIR, exist_ok=True)
    stamp = _LIB + ".flags"
    flags = "gcc -O3 -std=c11"
    if (not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.exists(stamp) and open(stamp).read() == flags):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    with open(stamp, "w") as f:
        f.write(flags)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(ctypes.c_double)
        PI = ctypes.POINTER(ctypes.c_int)
        PL = ctypes.POINTER(ctypes.c_int64)
        i, d = ctypes.c_int, ctypes.c_double
        L.oracle_build_schur.argtypes = [i, i, i, P, P, P, P, P, P, P]
        L.oracle_build_schur_full.argtypes = [i, i, i, P, P, P, P, P, P, P]
        L.oracle_build_precond.argtypes = [i, i, i, P, P, P, P, P, P]
        L.oracle_pcg.argtypes = [i, i, P, P, P, P, P, P, P, P, i, d, i, PI, P, P]
        L.oracle_pcg_poly.argtypes = [i, i, P, P, P, P, P, P, i, P, P, i, d, i, PI, P, P]
        L.oracle_apply_poly.argtypes = [i, i, P, P, P, P, P, P, i, P, P]
        L.oracle_solve_batch.argtypes = [i, PI, PI, PI, PL, PL, PL, PL, PL, P, P, P, P, P, i, d, i, P, PI, P, PI, i]
        L.oracle_solve_batch_poly.argtypes = [i, PI, PI, PI, PL, PL, PL, PL, PL, P, P, P, P, P, i, i, d, i, P, PI, P,
                                              PI, i]
        for f in (L.oracle_build_schur, L.oracle_build_schur_full, L.oracle_build_precond, L.oracle_pcg, L.oracle_pcg_poly,
                  L.oracle_apply_poly, L.oracle_solve_batch, L.oracle_solve_batch_poly):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class BlockTridiag:
    """d[k] = M(k,k), l[k] = M(k,k-1), u[k] = M(k,k+1); arrays [N+1, nx, nx]."""

    def __init__(self, d, l, u):
        self.d, self.l, self.u = d, l, u

    @property
    def N(self):
        return self.d.shape[0] - 1

    @property
    def nx(self):
        return self.d.shape[1]

    def dense(self) -> np.ndarray:
        n, m = self.d.shape[0], self.d.shape[1]
        M = np.zeros((n * m, n * m))
        for k in range(n):
            M[k * m:(k + 1) * m, k * m:(k + 1) * m] = self.d[k]
            if k > 0:
                M[k * m:(k + 1) * m, (k - 1) * m:k * m] = self.l[k]
            if k < n - 1:
                M[k * m:(k + 1) * m, (k + 1) * m:(k + 2) * m] = self.u[k]
        return M


def build_schur(A, B, qd, rd) -> BlockTridiag:
    A, B, qd, rd = _f64(A), _f64(B), _f64(qd), _f64(rd)
    N, nx = qd.shape[0] - 1, qd.shape[1]
    nu = rd.shape[1] if rd.ndim == 2 and N > 0 else (B.shape[2] if B.ndim == 3 else 0)
    d = np.zeros((N + 1, nx, nx)); l = np.zeros_like(d); u = np.zeros_like(d)
    rc = lib().oracle_build_schur(N, nx, nu, _p(A), _p(B), _p(qd), _p(rd), _p(d), _p(l), _p(u))
    if rc != OK:
        raise ValueError(f"oracle_build_schur failed: {rc}")
    return BlockTridiag(d, l, u)


def build_schur_full(A, B, Q, R) -> BlockTridiag:
    """S with full SPD cost blocks Q [N+1][nx][nx], R [N][nu][nu] (Sec. II-A formulas with matrix inverses)."""
    A, B, Q = _f64(A), _f64(B), _f64(Q)
    N, nx = Q.shape[0] - 1, Q.shape[1]
    nu = B.shape[2] if N > 0 and B.ndim == 3 else 0
    R = _f64(R).reshape(N, nu, nu) if N > 0 and nu > 0 else np.zeros(1)
    A = A if A.size else np.zeros(1)
    B = B if B.size else np.zeros(1)
    d = np.zeros((N + 1, nx, nx)); l = np.zeros_like(d); u = np.zeros_like(d)
    rc = lib().oracle_build_schur_full(N, nx, nu, _p(A), _p(B), _p(Q), _p(R), _p(d), _p(l), _p(u))
    if rc == NOT_SPD:
        raise np.linalg.LinAlgError("cost block not positive definite")
    if rc != OK:
        raise ValueError(f"oracle_build_schur_full failed: {rc}")
    return BlockTridiag(d, l, u)


def build_precond(S: BlockTridiag, kind: str | int = "sym") -> BlockTridiag:
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    d = np.zeros_like(S.d); l = np.zeros_like(S.d); u = np.zeros_like(S.d)
    rc = lib().oracle_build_precond(S.N, S.nx, k, _p(S.d), _p(S.l), _p(S.u), _p(d), _p(l), _p(u))
    if rc == NOT_SPD:
        raise np.linalg.LinAlgError("diagonal block not positive definite")
    if rc != OK:
        raise ValueError(f"oracle_build_precond failed: {rc}")
    return BlockTridiag(d, l, u)


def pcg(S: BlockTridiag, M: BlockTridiag, gamma, tol: float, max_iter: int | None = None, x0=None, degree: int = 0):
    """Returns (x [N+1, nx], iters, relres, true_relres, status).  degree > 0: the degree-d polynomial
    preconditioner of the splitting S = Psi - P with Psi^-1 = M (Eq. polynomial_precon)."""
    g = _f64(gamma).reshape(S.N + 1, S.nx)
    x = np.zeros_like(g) if x0 is None else _f64(x0).reshape(g.shape).copy()
    it = ctypes.c_int(0); rr = ctypes.c_double(0); tr = ctypes.c_double(0)
    mi = 10 * (S.N + 1) * S.nx if max_iter is None else int(max_iter)
    st = lib().oracle_pcg_poly(S.N, S.nx, _p(S.d), _p(S.l), _p(S.u), _p(M.d), _p(M.l), _p(M.u), int(degree), _p(g),
                               _p(x), 0 if x0 is None else 1, float(tol), mi, ctypes.byref(it), ctypes.byref(rr),
                               ctypes.byref(tr))
    return x, it.value, rr.value, tr.value, st


def apply_poly(S: BlockTridiag, M: BlockTridiag, degree: int, r) -> np.ndarray:
    """z = sum_{j<=degree} (Psi^-1 P)^j Psi^-1 r with Psi^-1 = M, P = Psi - S (Eq. polynomial_precon)."""
    r = _f64(r).reshape(S.N + 1, S.nx)
    z = np.zeros_like(r)
    rc = lib().oracle_apply_poly(S.N, S.nx, _p(S.d), _p(S.l), _p(S.u), _p(M.d), _p(M.l), _p(M.u), int(degree), _p(r),
                                 _p(z))
    if rc != OK:
        raise ValueError(f"oracle_apply_poly failed: {rc}")
    return z


def solve_problem(p, kind="sym", tol=1e-6, max_iter=None, x0=None, degree=0):
    """Whole path for one ``problems.Problem``: returns (S, M, x, iters, relres, true_relres, status)."""
    S = build_schur(p.A, p.B, p.qd, p.rd)
    M = build_precond(S, kind)
    x, it, rr, tr, st = pcg(S, M, p.gamma, tol, max_iter, x0, degree)
    return S, M, x, it, rr, tr, st


def solve_batch(problems, kind="sym", tol=1e-6, max_iter=0, nthreads=0, degree=0):
    """Whole path for a list of problems (OpenMP over problems).

    Returns (list of x arrays, iters, relres, status, threads_used, seconds).
    """
    nprob = len(problems)
    Ns = np.array([p.N for p in problems], dtype=np.int32)
    nxs = np.array([p.nx for p in problems], dtype=np.int32)
    nus = np.array([p.nu for p in problems], dtype=np.int32)

    def pack(arrs):
        sizes = np.array([a.size for a in arrs], dtype=np.int64)
        offs = np.zeros(nprob, dtype=np.int64)
        offs[1:] = np.cumsum(sizes)[:-1]
        flat = np.concatenate([a.ravel().astype(np.float64) for a in arrs]) if nprob else np.zeros(0)
        return np.ascontiguousarray(flat), offs

    A, oA = pack([p.A for p in problems]); B, oB = pack([p.B for p in problems])
    q, oq = pack([p.qd for p in problems]); r, orr = pack([p.rd for p in problems])
    g, og = pack([p.gamma for p in problems])
    # keep every pointer valid even for empty arrays
    A, B, r = (a if a.size else np.zeros(1) for a in (A, B, r))
    x = np.zeros_like(g)
    iters = np.zeros(nprob, dtype=np.int32); relres = np.zeros(nprob); status = np.zeros(nprob, dtype=np.int32)
    PI = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    PL = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    t0 = time.perf_counter()
    used = lib().oracle_solve_batch_poly(nprob, PI(Ns), PI(nxs), PI(nus), PL(oA), PL(oB), PL(oq), PL(orr), PL(og),
                                         _p(A), _p(B), _p(q), _p(r), _p(g), k, int(degree), float(tol),
                                         int(max_iter), _p(x), PI(iters), _p(relres), PI(status), int(nthreads))
    dt = time.perf_counter() - t0
    xs = [x[og[i]:og[i] + problems[i].gamma.size].reshape(problems[i].gamma.shape) for i in range(nprob)]
    return xs, iters, relres, status, used, dt
