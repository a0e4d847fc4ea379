"""Seeded synthetic trajectory-optimisation QPs (inputs only).

This module draws the per-knot data of the equality-constrained QP of
Sec. II-A (dynamics Jacobians A_k, B_k, diagonal cost Hessians Q_k, R_k and
the right-hand side gamma).  It holds none of the method's arithmetic: no
Schur complement, no preconditioner, no solver.  Both the CUDA path and the
FP64 oracle are fed from here, so that the two see bit-identical inputs.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
j-th 64-bit draw of stream ``key`` is ``mix(key + j * 0x9E3779B97F4A7C15)``
for j = 1, 2, ...  Uniforms take the top 53 bits; normals use the Box-Muller
transform on consecutive uniform pairs.

Per-problem draw order (stream key = config * 2**32 + index):
  draws 0, 1          shape uniforms (horizon N and state size nx, batched
                      workloads only)
  normals             G (N*nx*nx, scaled by 1/sqrt(nx)), B (N*nx*nu, scaled
                      by h), gamma ((N+1)*nx), Box-Muller pairs from draw 2
  uniforms            diag Q ((N+1)*nx, U[0.1, 10]), diag R (N*nu, U[0.1, 1])

A_k = I + h*G_k with G_k ~ N(0, 1/nx) is the integrator form of Sec. II-A
(A = I + hM, B = hN).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterable, List, Sequence

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start+1 .. start+count of the SplitMix64 stream ``key`` (uint64)."""
    j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + j * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(key: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(key, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(key: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` standard normals by Box-Muller, using 2*ceil(count/2) draws."""
    pairs = (count + 1) // 2
    u = uniform01(key, 2 * pairs, start)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    rho = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * pairs, dtype=np.float64)
    out[0::2] = rho * np.cos(2.0 * np.pi * u2)
    out[1::2] = rho * np.sin(2.0 * np.pi * u2)
    return out[:count]


def nu_for(nx: int) -> int:
    """Input size rule of the batched workloads: nx/2 rounded half up."""
    return (nx + 1) // 2


@dataclasses.dataclass
class Problem:
    """One QP instance.  Arrays are float32, row-major.

    A: [N, nx, nx]   B: [N, nx, nu]   qd: [N+1, nx]   rd: [N, nu]
    gamma: [N+1, nx] (right-hand side of the Schur system)
    """

    N: int
    nx: int
    nu: int
    A: np.ndarray
    B: np.ndarray
    qd: np.ndarray
    rd: np.ndarray
    gamma: np.ndarray
    key: int = 0

    @property
    def n(self) -> int:
        return self.N + 1


def make_problem(key: int, N: int, nx: int, nu: int, h: float) -> Problem:
    """Draw one problem of the given shape from stream ``key``."""
    if N < 0 or nx < 1 or nu < 0:
        raise ValueError("bad problem shape")
    n_g, n_b, n_gam = N * nx * nx, N * nx * nu, (N + 1) * nx
    n_norm = n_g + n_b + n_gam
    z = normals(key, n_norm, start=2)
    G = z[:n_g].reshape(N, nx, nx) / math.sqrt(nx)
    A = np.eye(nx)[None, :, :] + h * G
    B = h * z[n_g:n_g + n_b].reshape(N, nx, nu)
    gamma = z[n_g + n_b:].reshape(N + 1, nx)
    ustart = 2 + 2 * ((n_norm + 1) // 2)
    u = uniform01(key, (N + 1) * nx + N * nu, start=ustart)
    qd = (0.1 + 9.9 * u[:(N + 1) * nx]).reshape(N + 1, nx)
    rd = (0.1 + 0.9 * u[(N + 1) * nx:]).reshape(N, nu)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Problem(N, nx, nu, f32(A), f32(B), f32(qd), f32(rd), f32(gamma), key)


def config_key(config: int, index: int) -> int:
    return (config << 32) + index


# ---------------------------------------------------------------------------
# Named workloads.  Each returns the problem shapes and the generator settings.
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    config: int
    nprob: int
    h: float
    tol: float
    N_range: tuple | None = None      # inclusive (lo, hi) for batched draws
    nx_set: tuple | None = None       # choice set for nx
    nx_range: tuple | None = None     # inclusive (lo, hi) for nx
    N_fixed: int | None = None
    nx_fixed: int | None = None
    nu_fixed: int | None = None
    index_base: int = 0


PENDULUM_SINGLE = Workload("pendulum-like single solve nx=2 nu=1 N=20", 1, 1, 0.05, 1e-8,
                           N_fixed=20, nx_fixed=2, nu_fixed=1)
MANIPULATOR_SINGLE = Workload("manipulator-like single solve nx=14 nu=7 N=64", 2, 1, 0.01, 1e-6,
                              N_fixed=64, nx_fixed=14, nu_fixed=7)
RAGGED_BATCH_4096 = Workload("ragged batch 4096 problems N~U{16..128} nx in {4,12,14,21}", 3, 4096,
                             0.05, 1e-6, N_range=(16, 128), nx_set=(4, 12, 14, 21))
WARMSTART_EVAL_4096 = Workload("warm-start eval 4096 problems nx=14 nu=7 N=64", 4, 4096, 0.01, 1e-6,
                               N_fixed=64, nx_fixed=14, nu_fixed=7, index_base=10 ** 9)
MPC_BATCH_16384 = Workload("MPC batch 16384 problems N~U{64..512} nx~U{4..28}", 5, 16384, 0.05, 1e-6,
                           N_range=(64, 512), nx_range=(4, 28))

# many small problems (more than the GPU holds at once at one problem per CTA): the case for one problem per warp
SMALL_BATCH_16384 = Workload("small batch 16384 problems N~U{8..32} nx in {2,4,6}", 6, 16384, 0.05, 1e-6,
                             N_range=(8, 32), nx_set=(2, 4, 6))
WORKLOADS = {w.config: w for w in (PENDULUM_SINGLE, MANIPULATOR_SINGLE, RAGGED_BATCH_4096,
                                   WARMSTART_EVAL_4096, MPC_BATCH_16384, SMALL_BATCH_16384)}


def problem_shape(w: Workload, index: int) -> tuple:
    """(key, N, nx, nu) of problem ``index`` of workload ``w``."""
    key = config_key(w.config, w.index_base + index)
    u = uniform01(key, 2, 0)
    if w.N_fixed is not None:
        N = w.N_fixed
    else:
        lo, hi = w.N_range
        N = lo + int(u[0] * (hi - lo + 1))
    if w.nx_fixed is not None:
        nx = w.nx_fixed
    elif w.nx_set is not None:
        nx = w.nx_set[int(u[1] * len(w.nx_set))]
    else:
        lo, hi = w.nx_range
        nx = lo + int(u[1] * (hi - lo + 1))
    nu = w.nu_fixed if w.nu_fixed is not None else nu_for(nx)
    return key, N, nx, nu


def make_workload(w: Workload, count: int | None = None, start: int = 0) -> List[Problem]:
    """Problems start .. start+count-1 of workload ``w`` (all of them by default)."""
    count = w.nprob - start if count is None else count
    out = []
    for i in range(start, start + count):
        key, N, nx, nu = problem_shape(w, i)
        out.append(make_problem(key, N, nx, nu, w.h))
    return out


def perturb_gamma(p: Problem, resolve: int, rel: float = 0.01) -> np.ndarray:
    """gamma * (1 + rel * xi) for the ``resolve``-th sequential re-solve (MPC workload).

    xi ~ N(0, 1) per entry, drawn from a stream of its own
    (problem key + (resolve+1) * 2**48).
    """
    key = p.key + ((resolve + 1) << 48)
    xi = normals(key, p.gamma.size, 0).reshape(p.gamma.shape)
    return (p.gamma.astype(np.float64) * (1.0 + rel * xi)).astype(np.float32)


def custom_problems(shapes: Iterable[Sequence[int]], h: float = 0.05, config: int = 99) -> List[Problem]:
    """Problems of explicit shapes (N, nx[, nu]) for tests; keys config*2**32 + i."""
    out = []
    for i, s in enumerate(shapes):
        N, nx = int(s[0]), int(s[1])
        nu = int(s[2]) if len(s) > 2 else nu_for(nx)
        out.append(make_problem(config_key(config, i), N, nx, nu, h))
    return out


# ---------------------------------------------------------------------------
# Warm-start network: seeded initial weights (inputs, like the problems).
# ---------------------------------------------------------------------------
MLP_SHAPES = ((256, 1344), (256,), (256, 256), (256,), (32, 256), (32,))


def mlp_initial_params(seed: int = 0) -> np.ndarray:
    """Flat FP32 initial parameters [W1, b1, W2, b2, W3, b3] of the warm-start network.

    W1 and W2 ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from stream ``2**62 + seed``
    (W1 first, then W2); biases zero; the output layer W3, b3 zero, so that the
    untrained network predicts lambda0 = 0 (the plain method's start)."""
    key = (1 << 62) + seed
    n1, n2 = 256 * 1344, 256 * 256
    u = uniform01(key, n1 + n2, 0)
    w1 = (2.0 * u[:n1] - 1.0) / math.sqrt(1344)
    w2 = (2.0 * u[n1:] - 1.0) / math.sqrt(256)
    parts = [w1, np.zeros(256), w2, np.zeros(256), np.zeros(32 * 256), np.zeros(32)]
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


def _chunk(args):
    config, count, start = args
    return make_workload(WORKLOADS[config], count=count, start=start)


def make_workload_parallel(w: Workload, count: int | None = None, start: int = 0, workers: int | None = None,
                           chunk: int = 256) -> List[Problem]:
    """``make_workload`` split over a pool of spawned processes (the same problems, in order).  Spawned, not
    forked, so that it is safe after the parent has initialised CUDA."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    count = w.nprob - start if count is None else count
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or count <= chunk:
        return make_workload(w, count, start)
    jobs = [(w.config, min(chunk, count - i), start + i) for i in range(0, count, chunk)]
    out: List[Problem] = []
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for part in ex.map(_chunk, jobs):
            out.extend(part)
    return out


def qp_vectors(p: Problem, seed: int = 0):
    """Constraint values c [N+1, nx] and cost gradients q [N+1, nx], r [N, nu] of problem ``p`` (FP32),
    N(0, 1) entries from stream ``p.key + (seed + 1) * 2**56`` in the order c, q, r."""
    n, m, u = p.N + 1, p.nx, p.nu
    z = normals(p.key + ((seed + 1) << 56), 2 * n * m + p.N * u, 0)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return (f32(z[:n * m].reshape(n, m)), f32(z[n * m:2 * n * m].reshape(n, m)),
            f32(z[2 * n * m:].reshape(p.N, u)))


def full_cost(p: Problem, seed: int = 0):
    """Full SPD cost blocks of problem ``p`` (FP32, exactly symmetric):
    Q_k = diag(qd_k) + M_k M_k^T / nx  [N+1, nx, nx],  R_k = diag(rd_k) + W_k W_k^T / nu  [N, nu, nu],
    M_k, W_k with N(0, 1) entries from stream ``p.key + (seed + 1) * 2**52`` (all M_k, then all W_k).
    The diagonal of p is kept, so Q_k >= diag(qd_k) and the coupling is of the same size."""
    n, m, u = p.N + 1, p.nx, p.nu
    z = normals(p.key + ((seed + 1) << 52), n * m * m + p.N * u * u, 0)
    M = z[:n * m * m].reshape(n, m, m)
    W = z[n * m * m:].reshape(p.N, u, u)
    Q = np.einsum("kij,klj->kil", M, M) / m + np.einsum("ki,ij->kij", p.qd.astype(np.float64), np.eye(m))
    R = (np.einsum("kij,klj->kil", W, W) / max(u, 1) +
         np.einsum("ki,ij->kij", p.rd.astype(np.float64), np.eye(u))) if p.N > 0 else np.zeros((0, u, u))
    sym = lambda a: np.ascontiguousarray((a + np.swapaxes(a, 1, 2)) * 0.5, dtype=np.float32)
    return sym(Q), sym(R)
