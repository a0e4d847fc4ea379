"""Python binding of the sspcg C ABI (``include/sspcg.h``).

Argument marshalling only: every step of the path runs in the CUDA library.
Functions carry the C names and take torch CUDA tensors for device arrays;
``stream`` defaults to torch's current stream.  Any non-OK return raises.
The library must have been built (``paper_2309_06427_gb300.build.build()``);
loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA = 0, 1, 2, 3
SOLVE_OK, SOLVE_MAXITER, SOLVE_BREAKDOWN, SOLVE_NOT_SPD, SOLVE_NONFINITE = 0, 1, 2, 3, 4
PRECOND = {"sym": 0, "add": 1, "bj": 2, "jacobi": 3}
REDUCE = {"df": 0, "f32": 1, "f64": 2}
SCHED = {"auto": 0, "resident": 1, "stream": 2, "warp": 3}
PRECISION = {"auto": 0, "f32": 1, "f64": 2}
ARRAY_A, ARRAY_B, ARRAY_QD, ARRAY_RD, ARRAY_DIAG, ARRAY_OFF, ARRAY_VEC, ARRAY_RFULL = range(8)
NUM_ARRAYS = 8
MAX_NX = 28
NOALLOC_MAX_PROBLEMS = 4096


class SspcgError(RuntimeError):
    pass


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("reduction", ctypes.c_int32), ("schedule", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("poly_degree", ctypes.c_int32), ("cg_variant", ctypes.c_int32)]


MAX_POLY_DEGREE = 16


def options(tol=1e-6, max_iter=0, warm_start=0, reduction="df", schedule="auto", block_threads=0,
            precision="auto", poly_degree=0, cg_variant=0) -> Options:
    pick = lambda table, v: table[v] if isinstance(v, str) else int(v)
    return Options(float(tol), int(max_iter), int(warm_start), pick(REDUCE, reduction), pick(SCHED, schedule),
                   int(block_threads), pick(PRECISION, precision), int(poly_degree), int(cg_variant))


_lib = None
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


def adam(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> Adam:
    return Adam(lr, beta1, beta2, eps)


MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 1344, 256, 32, 418336


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise SspcgError(f"sspcg CUDA library missing at {_build.LIB}; build it with "
                             "paper_2309_06427_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(_build.LIB)
        sig = {
            "sspcg_build_schur": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_build_precond": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_solve": [_I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(Options), _VP, _VP, _VP, _VP],
            "sspcg_solve_qp": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(Options),
                               _VP, _VP, _VP, _VP],
            "sspcg_residual_qp": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_build_schur_f64": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_build_precond_f64": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_solve_qp_f64": [_I32, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(Options),
                                   _VP, _VP, _VP, _VP],
            "sspcg_plan_create": [ctypes.POINTER(_VP), _I32, _VP, _VP, _VP, ctypes.POINTER(Options)],
            "sspcg_plan_destroy": [_VP],
            "sspcg_plan_sizes": [_VP, _VP],
            "sspcg_plan_offsets": [_VP, _I32, _VP],
            "sspcg_plan_stats": [_VP, _VP],
            "sspcg_plan_set_timing": [_VP, _I32],
            "sspcg_plan_timings": [_VP, _VP],
            "sspcg_plan_capture_pipeline": [_VP, _I32] + [_VP] * 14,
            "sspcg_plan_launch": [_VP, _VP],
            "sspcg_build_schur_batched": [_VP] * 8,
            "sspcg_schur_full_work_floats": [_I32, _I32, _I32, _VP],
            "sspcg_build_schur_full": [_I32, _I32, _I32] + [_VP] * 9,
            "sspcg_build_schur_full_batched": [_VP] * 9,
            "sspcg_build_precond_batched": [_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP],
            "sspcg_solve_batched": [_VP] * 11,
            "sspcg_solve_qp_batched": [_VP] * 13,
            "sspcg_residual_qp_batched": [_VP] * 9,
            "sspcg_pipeline_batched": [_VP, _I32] + [_VP] * 14,
            "sspcg_pipeline_host": [_VP, _I32] + [_VP] * 10,
            "sspcg_pipeline_host_async": [_VP, _I32] + [_VP] * 10,
            "sspcg_plan_join": [_VP, _VP],
            "sspcg_solve_qp_batched_noalloc": [_I32] + [_VP] * 11 + [ctypes.POINTER(Options)] + [_VP] * 4,
            "sspcg_mlp_create": [ctypes.POINTER(_VP), _I32],
            "sspcg_mlp_destroy": [_VP],
            "sspcg_mlp_set_params": [_VP, _VP, _VP],
            "sspcg_mlp_set_engine": [_VP, _I32],
            "sspcg_mlp_status": [_VP, _VP],
            "sspcg_mlp_get_params": [_VP, _VP, _VP],
            "sspcg_mlp_get_grads": [_VP, _VP, _VP],
            "sspcg_mlp_set_normalisation": [_VP, _VP, _VP, _VP],
            "sspcg_mlp_get_normalisation": [_VP, _VP, _VP, _VP],
            "sspcg_mlp_fit_normalisation": [_VP] * 9,
            "sspcg_mlp_features": [_VP, _VP, _I32, _I32] + [_VP] * 8,
            "sspcg_mlp_infer": [_VP] * 10,
            "sspcg_mlp_train_step": [_VP, _VP, _I32, _I32] + [_VP] * 9 + [ctypes.POINTER(Adam), _VP, _VP],
            "sspcg_pipeline_warm_batched": [_VP, _VP, _I32] + [_VP] * 14,
            "sspcg_form_gamma": [_I32, _I32, _I32] + [_VP] * 9,
            "sspcg_recover_step": [_I32, _I32, _I32] + [_VP] * 10,
            "sspcg_form_gamma_batched": [_VP] * 10,
            "sspcg_recover_step_batched": [_VP] * 11,
            "sspcg_measure_smem_bandwidth": [_I32, _I32, _VP, _VP],
            "sspcg_mlp_checkpoint_bytes": [_VP],
            "sspcg_plan_autotune": [_VP, _I32, _I32] + [_VP] * 14,
            "sspcg_plan_schedule": [_VP, _I32, _VP, _I32, _VP],
            "sspcg_autotune_cache_clear": [],
            "sspcg_mlp_save": [_VP, _VP, ctypes.c_int64, _VP],
            "sspcg_mlp_load": [_VP, _VP, ctypes.c_int64, _VP],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sspcg_last_cuda_error.restype = ctypes.c_char_p
        L.sspcg_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return [n for n in dir(lib()) if n.startswith("sspcg_")]


def _check(rc: int, what: str):
    if rc != OK:
        msg = {ERR_INVALID_ARG: "invalid argument", ERR_UNSUPPORTED: "unsupported",
               ERR_CUDA: "CUDA error: " + lib().sspcg_last_cuda_error().decode()}.get(rc, f"code {rc}")
        raise SspcgError(f"{what}: {msg}")


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise SspcgError("device tensor expected")
    if not t.is_contiguous():
        raise SspcgError("contiguous tensor expected")
    return t.data_ptr() or None


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# Single problem
# ---------------------------------------------------------------------------
def sspcg_build_schur(N, nx, nu, A, B, qd, rd, D, E, stream=None):
    _check(lib().sspcg_build_schur(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(D), _ptr(E),
                                   _stream(stream)), "sspcg_build_schur")


def sspcg_build_precond(N, nx, kind, D, E, PD, PE, status, stream=None):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_build_precond(N, nx, k, _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(status),
                                     _stream(stream)), "sspcg_build_precond")


def sspcg_solve(N, nx, D, E, PD, PE, gamma, lam, opts: Options, iters, relres, status, stream=None):
    _check(lib().sspcg_solve(N, nx, _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(gamma), _ptr(lam),
                             ctypes.byref(opts), _ptr(iters), _ptr(relres), _ptr(status), _stream(stream)),
           "sspcg_solve")


def sspcg_solve_qp(N, nx, nu, A, B, qd, rd, PD, PE, gamma, lam, opts: Options, iters, relres, status, stream=None):
    _check(lib().sspcg_solve_qp(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(PD), _ptr(PE), _ptr(gamma),
                                _ptr(lam), ctypes.byref(opts), _ptr(iters), _ptr(relres), _ptr(status),
                                _stream(stream)), "sspcg_solve_qp")


def sspcg_build_schur_f64(N, nx, nu, A, B, qd, rd, D, E, stream=None):
    _check(lib().sspcg_build_schur_f64(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(D), _ptr(E),
                                       _stream(stream)), "sspcg_build_schur_f64")


def sspcg_build_precond_f64(N, nx, kind, D, E, PD, PE, status, stream=None):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_build_precond_f64(N, nx, k, _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(status),
                                         _stream(stream)), "sspcg_build_precond_f64")


def sspcg_solve_qp_f64(N, nx, nu, A, B, qd, rd, PD, PE, gamma, lam, opts: Options, iters, relres, status,
                       stream=None):
    _check(lib().sspcg_solve_qp_f64(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(PD), _ptr(PE),
                                    _ptr(gamma), _ptr(lam), ctypes.byref(opts), _ptr(iters), _ptr(relres),
                                    _ptr(status), _stream(stream)), "sspcg_solve_qp_f64")


def sspcg_residual_qp(N, nx, nu, A, B, qd, rd, gamma, lam, relres_true, stream=None):
    _check(lib().sspcg_residual_qp(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma), _ptr(lam),
                                   _ptr(relres_true), _stream(stream)), "sspcg_residual_qp")


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------
class Plan:
    """Owner of an ``sspcg_plan``; destroyed with the object."""

    def __init__(self, N: Sequence[int], nx: Sequence[int], nu: Sequence[int], opts: Options):
        self.N = np.ascontiguousarray(N, dtype=np.int32)
        self.nx = np.ascontiguousarray(nx, dtype=np.int32)
        self.nu = np.ascontiguousarray(nu, dtype=np.int32)
        self.nprob = len(self.N)
        self.opts = opts
        h = _VP()
        _check(lib().sspcg_plan_create(ctypes.byref(h), self.nprob, self.N.ctypes.data, self.nx.ctypes.data,
                                       self.nu.ctypes.data, ctypes.byref(opts)), "sspcg_plan_create")
        self.handle = h
        sizes = np.zeros(NUM_ARRAYS, dtype=np.int64)
        _check(lib().sspcg_plan_sizes(h, sizes.ctypes.data), "sspcg_plan_sizes")
        self.sizes = sizes
        self.offsets = []
        for k in range(NUM_ARRAYS):
            o = np.zeros(self.nprob, dtype=np.int64)
            if self.nprob:
                _check(lib().sspcg_plan_offsets(h, k, o.ctypes.data), "sspcg_plan_offsets")
            self.offsets.append(o)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.sspcg_plan_destroy(h)
            self.handle = None

    def empty(self, kind: int, device="cuda", dtype=torch.float32, fill=0.0) -> torch.Tensor:
        return torch.full((max(int(self.sizes[kind]), 4),), fill, dtype=dtype, device=device)

    def pack(self, kind: int, arrays: Sequence[np.ndarray], out: Optional[np.ndarray] = None) -> np.ndarray:
        """Pack per-problem arrays (host) into the plan's layout (host float32)."""
        flat = np.zeros(max(int(self.sizes[kind]), 4), dtype=np.float32) if out is None else out
        offs = self.offsets[kind]
        for i, a in enumerate(arrays):
            a = np.asarray(a, dtype=np.float32).ravel()
            flat[offs[i]:offs[i] + a.size] = a
        return flat

    def unpack(self, kind: int, flat, shapes: Sequence[tuple]) -> List[np.ndarray]:
        flat = flat.detach().cpu().numpy() if isinstance(flat, torch.Tensor) else np.asarray(flat)
        offs = self.offsets[kind]
        out = []
        for i, shp in enumerate(shapes):
            n = int(np.prod(shp))
            out.append(flat[offs[i]:offs[i] + n].reshape(shp))
        return out


def sspcg_plan_create(N, nx, nu, opts: Options) -> Plan:
    return Plan(N, nx, nu, opts)


def sspcg_plan_stats(plan: Plan) -> Dict[str, int]:
    out = np.zeros(8, dtype=np.int64)
    _check(lib().sspcg_plan_stats(plan.handle, out.ctypes.data), "sspcg_plan_stats")
    keys = ["pipeline_launches", "pipeline_resident", "pipeline_stream", "pipeline_f64", "solve_qp_launches",
            "solve_block_launches", "solve_qp_resident", "solve_qp_stream"]
    return {k: int(v) for k, v in zip(keys, out)}


def sspcg_plan_set_timing(plan: Plan, enable: bool = True):
    _check(lib().sspcg_plan_set_timing(plan.handle, int(bool(enable))), "sspcg_plan_set_timing")


def sspcg_plan_timings(plan: Plan):
    """(build_ms, pcg_ms) of the plan's last pipeline or solve call."""
    out = np.zeros(2, dtype=np.float32)
    _check(lib().sspcg_plan_timings(plan.handle, out.ctypes.data), "sspcg_plan_timings")
    return float(out[0]), float(out[1])


def sspcg_plan_capture_pipeline(plan: Plan, kind, A, B, qd, rd, gamma, D, E, PD, PE, lam, iters, relres, status,
                                stream):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_plan_capture_pipeline(plan.handle, k, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma),
                                             _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(lam), _ptr(iters),
                                             _ptr(relres), _ptr(status), _stream(stream)),
           "sspcg_plan_capture_pipeline")


def sspcg_plan_autotune(plan: Plan, kind, A, B, qd, rd, gamma, D, E, PD, PE, lam, iters, relres, status, stream=None,
                        which="all"):
    """Tune the plan's PCG launch groups on these inputs: which = "pipeline", "solve" or "all"."""
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    wh = {"pipeline": 1, "solve": 2, "all": 3}[which]
    _check(lib().sspcg_plan_autotune(plan.handle, wh, k, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma),
                                     _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(lam), _ptr(iters), _ptr(relres),
                                     _ptr(status), _stream(stream)), "sspcg_plan_autotune")


SCHEDULE_FIELDS = ("nx", "cls", "problems", "max_N", "block", "grid", "smem", "stream", "tuned", "share", "warps")


def sspcg_plan_schedule(plan: Plan, which: str = "pipeline") -> List[Dict[str, int]]:
    """Launch groups of a plan: which = "pipeline" (FP32 set), "pipeline_f64" or "solve_qp"."""
    w = {"pipeline": 0, "pipeline_f64": 1, "solve_qp": 2}[which]
    cnt = ctypes.c_int32(0)
    _check(lib().sspcg_plan_schedule(plan.handle, w, None, 0, ctypes.addressof(cnt)), "sspcg_plan_schedule")
    out = np.zeros((max(cnt.value, 1), len(SCHEDULE_FIELDS)), dtype=np.int32)
    _check(lib().sspcg_plan_schedule(plan.handle, w, out.ctypes.data, cnt.value, ctypes.addressof(cnt)),
           "sspcg_plan_schedule")
    return [dict(zip(SCHEDULE_FIELDS, map(int, row))) for row in out[:cnt.value]]


def sspcg_autotune_cache_clear():
    _check(lib().sspcg_autotune_cache_clear(), "sspcg_autotune_cache_clear")


def sspcg_plan_launch(plan: Plan, stream=None):
    _check(lib().sspcg_plan_launch(plan.handle, _stream(stream)), "sspcg_plan_launch")


plan_stats = sspcg_plan_stats


def sspcg_build_schur_batched(plan: Plan, A, B, qd, rd, D, E, stream=None):
    _check(lib().sspcg_build_schur_batched(plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(D), _ptr(E),
                                           _stream(stream)), "sspcg_build_schur_batched")


def sspcg_schur_full_work_floats(N, nx, nu) -> int:
    out = ctypes.c_int64(0)
    _check(lib().sspcg_schur_full_work_floats(N, nx, nu, ctypes.byref(out)), "sspcg_schur_full_work_floats")
    return int(out.value)


def sspcg_build_schur_full(N, nx, nu, A, B, Q, R, D, E, work, status, stream=None):
    """Schur blocks from full SPD Q_k, R_k (Sec. II-A); status: device int32[1]."""
    _check(lib().sspcg_build_schur_full(N, nx, nu, _ptr(A), _ptr(B), _ptr(Q), _ptr(R), _ptr(D), _ptr(E), _ptr(work),
                                        _ptr(status), _stream(stream)), "sspcg_build_schur_full")


def sspcg_build_schur_full_batched(plan: Plan, A, B, Q, R, D, E, status, stream=None):
    """Batched full-cost Schur build: Q packed like D (ARRAY_DIAG), R in ARRAY_RFULL."""
    _check(lib().sspcg_build_schur_full_batched(plan.handle, _ptr(A), _ptr(B), _ptr(Q), _ptr(R), _ptr(D), _ptr(E),
                                                _ptr(status), _stream(stream)), "sspcg_build_schur_full_batched")


def sspcg_build_precond_batched(plan: Plan, kind, D, E, PD, PE, status, stream=None):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_build_precond_batched(plan.handle, k, _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(status),
                                             _stream(stream)), "sspcg_build_precond_batched")


def sspcg_solve_batched(plan: Plan, D, E, PD, PE, gamma, lam, iters, relres, status, stream=None):
    _check(lib().sspcg_solve_batched(plan.handle, _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(gamma), _ptr(lam),
                                     _ptr(iters), _ptr(relres), _ptr(status), _stream(stream)),
           "sspcg_solve_batched")


def sspcg_solve_qp_batched(plan: Plan, A, B, qd, rd, PD, PE, gamma, lam, iters, relres, status, stream=None):
    _check(lib().sspcg_solve_qp_batched(plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(PD), _ptr(PE),
                                        _ptr(gamma), _ptr(lam), _ptr(iters), _ptr(relres), _ptr(status),
                                        _stream(stream)), "sspcg_solve_qp_batched")


def sspcg_residual_qp_batched(plan: Plan, A, B, qd, rd, gamma, lam, relres_true, stream=None):
    _check(lib().sspcg_residual_qp_batched(plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma),
                                           _ptr(lam), _ptr(relres_true), _stream(stream)),
           "sspcg_residual_qp_batched")


def sspcg_pipeline_batched(plan: Plan, kind, A, B, qd, rd, gamma, D, E, PD, PE, lam, iters, relres, status,
                           stream=None):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_pipeline_batched(plan.handle, k, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma), _ptr(D),
                                        _ptr(E), _ptr(PD), _ptr(PE), _ptr(lam), _ptr(iters), _ptr(relres),
                                        _ptr(status), _stream(stream)), "sspcg_pipeline_batched")


def sspcg_pipeline_host(plan: Plan, kind, A, B, qd, rd, gamma, lam, iters, relres, status, stream=None):
    """Host-buffer pipeline: A..gamma, lam, iters, relres, status are host torch tensors (pinned for speed)."""
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    hp = lambda t: t.data_ptr() if t is not None else None
    _check(lib().sspcg_pipeline_host(plan.handle, k, hp(A), hp(B), hp(qd), hp(rd), hp(gamma), hp(lam), hp(iters),
                                     hp(relres), hp(status), _stream(stream)), "sspcg_pipeline_host")


def sspcg_pipeline_host_async(plan: Plan, kind, A, B, qd, rd, gamma, lam, iters, relres, status, stream=None):
    """Host-buffer pipeline without the final wait (pinned host tensors; complete after sspcg_plan_join and a
    synchronisation of that stream)."""
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    hp = lambda t: t.data_ptr() if t is not None else None
    _check(lib().sspcg_pipeline_host_async(plan.handle, k, hp(A), hp(B), hp(qd), hp(rd), hp(gamma), hp(lam),
                                           hp(iters), hp(relres), hp(status), _stream(stream)),
           "sspcg_pipeline_host_async")


def sspcg_plan_join(plan: Plan, stream=None):
    _check(lib().sspcg_plan_join(plan.handle, _stream(stream)), "sspcg_plan_join")


def sspcg_solve_qp_batched_noalloc(N, nx, nu, A, B, qd, rd, PD, PE, gamma, lam, opts: Options, iters, relres, status,
                                   stream=None):
    """Batched FP32 solve without a plan and without any device allocation (shape arrays on the host)."""
    N = np.ascontiguousarray(N, dtype=np.int32)
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    nu = np.ascontiguousarray(nu, dtype=np.int32)
    _check(lib().sspcg_solve_qp_batched_noalloc(len(N), N.ctypes.data, nx.ctypes.data, nu.ctypes.data, _ptr(A),
                                                _ptr(B), _ptr(qd), _ptr(rd), _ptr(PD), _ptr(PE), _ptr(gamma),
                                                _ptr(lam), ctypes.byref(opts), _ptr(iters), _ptr(relres),
                                                _ptr(status), _stream(stream)), "sspcg_solve_qp_batched_noalloc")


# ---------------------------------------------------------------------------
# The QP step around the solve
# ---------------------------------------------------------------------------
def sspcg_measure_smem_bandwidth(load_bytes=16, rounds=4096, stream=None) -> float:
    """Measured shared-memory read bandwidth of the current device in GB/s (a diagnostic)."""
    out = ctypes.c_double(0.0)
    _check(lib().sspcg_measure_smem_bandwidth(int(load_bytes), int(rounds), ctypes.addressof(out), _stream(stream)),
           "sspcg_measure_smem_bandwidth")
    return out.value


def sspcg_form_gamma(N, nx, nu, A, B, qd, rd, c, q, r, gamma, stream=None):
    _check(lib().sspcg_form_gamma(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(c), _ptr(q), _ptr(r),
                                  _ptr(gamma), _stream(stream)), "sspcg_form_gamma")


def sspcg_recover_step(N, nx, nu, A, B, qd, rd, q, r, mu, dx, du, stream=None):
    _check(lib().sspcg_recover_step(N, nx, nu, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(q), _ptr(r), _ptr(mu),
                                    _ptr(dx), _ptr(du), _stream(stream)), "sspcg_recover_step")


def sspcg_form_gamma_batched(plan, A, B, qd, rd, c, q, r, gamma, stream=None):
    _check(lib().sspcg_form_gamma_batched(plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(c), _ptr(q),
                                          _ptr(r), _ptr(gamma), _stream(stream)), "sspcg_form_gamma_batched")


def sspcg_recover_step_batched(plan, A, B, qd, rd, q, r, mu, dx, du, stream=None):
    _check(lib().sspcg_recover_step_batched(plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(q), _ptr(r),
                                            _ptr(mu), _ptr(dx), _ptr(du), _stream(stream)),
           "sspcg_recover_step_batched")


# ---------------------------------------------------------------------------
# Learned warm start
# ---------------------------------------------------------------------------
class Mlp:
    """Owner of an ``sspcg_mlp`` network object (parameters, Adam state, workspace)."""

    def __init__(self, max_rows: int):
        h = _VP()
        _check(lib().sspcg_mlp_create(ctypes.byref(h), int(max_rows)), "sspcg_mlp_create")
        self.handle, self.max_rows = h, int(max_rows)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sspcg_mlp_destroy(self.handle)
            self.handle = None


def sspcg_mlp_create(max_rows: int) -> Mlp:
    return Mlp(max_rows)


MLP_ENGINE = {"tcgen05": 0, "mma_sync": 1}


def sspcg_mlp_set_engine(mlp: Mlp, engine="tcgen05"):
    e = MLP_ENGINE[engine] if isinstance(engine, str) else int(engine)
    _check(lib().sspcg_mlp_set_engine(mlp.handle, e), "sspcg_mlp_set_engine")


def sspcg_mlp_status(mlp: Mlp) -> int:
    v = ctypes.c_int32(0)
    _check(lib().sspcg_mlp_status(mlp.handle, ctypes.byref(v)), "sspcg_mlp_status")
    return int(v.value)


def sspcg_mlp_set_params(mlp: Mlp, params, stream=None):
    _check(lib().sspcg_mlp_set_params(mlp.handle, _ptr(params), _stream(stream)), "sspcg_mlp_set_params")


def sspcg_mlp_get_params(mlp: Mlp, params, stream=None):
    _check(lib().sspcg_mlp_get_params(mlp.handle, _ptr(params), _stream(stream)), "sspcg_mlp_get_params")


def sspcg_mlp_get_grads(mlp: Mlp, grads, stream=None):
    _check(lib().sspcg_mlp_get_grads(mlp.handle, _ptr(grads), _stream(stream)), "sspcg_mlp_get_grads")


def sspcg_mlp_checkpoint_bytes() -> int:
    out = ctypes.c_int64(0)
    _check(lib().sspcg_mlp_checkpoint_bytes(ctypes.addressof(out)), "sspcg_mlp_checkpoint_bytes")
    return out.value


def sspcg_mlp_save(mlp: Mlp, stream=None) -> np.ndarray:
    """Checkpoint of the network (parameters, Adam moments and step count, normalisation) as host bytes."""
    buf = np.zeros(sspcg_mlp_checkpoint_bytes(), dtype=np.uint8)
    _check(lib().sspcg_mlp_save(mlp.handle, buf.ctypes.data, buf.size, _stream(stream)), "sspcg_mlp_save")
    return buf


def sspcg_mlp_load(mlp: Mlp, buf, stream=None):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().sspcg_mlp_load(mlp.handle, buf.ctypes.data, buf.size, _stream(stream)), "sspcg_mlp_load")


def sspcg_mlp_set_normalisation(mlp: Mlp, mu, inv_sigma, stream=None):
    _check(lib().sspcg_mlp_set_normalisation(mlp.handle, _ptr(mu), _ptr(inv_sigma), _stream(stream)),
           "sspcg_mlp_set_normalisation")


def sspcg_mlp_get_normalisation(mlp: Mlp, mu, inv_sigma, stream=None):
    _check(lib().sspcg_mlp_get_normalisation(mlp.handle, _ptr(mu), _ptr(inv_sigma), _stream(stream)),
           "sspcg_mlp_get_normalisation")


def sspcg_mlp_fit_normalisation(mlp: Mlp, plan: Plan, A, B, qd, rd, gamma, PD, stream=None):
    _check(lib().sspcg_mlp_fit_normalisation(mlp.handle, plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd),
                                             _ptr(gamma), _ptr(PD), _stream(stream)), "sspcg_mlp_fit_normalisation")


def sspcg_mlp_features(mlp: Mlp, plan: Plan, p_begin, p_end, A, B, qd, rd, gamma, PD, X, stream=None):
    """X: device tensor (torch.bfloat16 or int16/uint16 bit patterns) of rows x MLP_IN."""
    _check(lib().sspcg_mlp_features(mlp.handle, plan.handle, int(p_begin), int(p_end), _ptr(A), _ptr(B), _ptr(qd),
                                    _ptr(rd), _ptr(gamma), _ptr(PD), _ptr(X), _stream(stream)), "sspcg_mlp_features")


def sspcg_mlp_infer(mlp: Mlp, plan: Plan, A, B, qd, rd, gamma, PD, lam0, stream=None):
    _check(lib().sspcg_mlp_infer(mlp.handle, plan.handle, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd), _ptr(gamma),
                                 _ptr(PD), _ptr(lam0), _stream(stream)), "sspcg_mlp_infer")


def sspcg_mlp_train_step(mlp: Mlp, plan: Plan, p_begin, p_end, A, B, qd, rd, gamma, D, E, PD, lam_star,
                         hyper: Adam, loss, stream=None):
    _check(lib().sspcg_mlp_train_step(mlp.handle, plan.handle, int(p_begin), int(p_end), _ptr(A), _ptr(B), _ptr(qd),
                                      _ptr(rd), _ptr(gamma), _ptr(D), _ptr(E), _ptr(PD), _ptr(lam_star),
                                      ctypes.byref(hyper), _ptr(loss), _stream(stream)), "sspcg_mlp_train_step")


def sspcg_pipeline_warm_batched(plan: Plan, mlp: Mlp, kind, A, B, qd, rd, gamma, D, E, PD, PE, lam, iters, relres,
                                status, stream=None):
    k = PRECOND[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sspcg_pipeline_warm_batched(plan.handle, mlp.handle, k, _ptr(A), _ptr(B), _ptr(qd), _ptr(rd),
                                             _ptr(gamma), _ptr(D), _ptr(E), _ptr(PD), _ptr(PE), _ptr(lam),
                                             _ptr(iters), _ptr(relres), _ptr(status), _stream(stream)),
           "sspcg_pipeline_warm_batched")


# ---------------------------------------------------------------------------
# Convenience: a packed batch of problems on the device
# ---------------------------------------------------------------------------
class Batch:
    """Packed device arrays of a list of ``problems.Problem`` for one plan."""

    def __init__(self, plan: Plan, probs, device="cuda", pin=False):
        self.plan, self.probs = plan, probs
        host = {
            "A": plan.pack(ARRAY_A, [p.A for p in probs]),
            "B": plan.pack(ARRAY_B, [p.B for p in probs]),
            "qd": plan.pack(ARRAY_QD, [p.qd for p in probs], np.ones(max(int(plan.sizes[ARRAY_QD]), 4), np.float32)),
            "rd": plan.pack(ARRAY_RD, [p.rd for p in probs], np.ones(max(int(plan.sizes[ARRAY_RD]), 4), np.float32)),
            "gamma": plan.pack(ARRAY_VEC, [p.gamma for p in probs]),
        }
        self.host = {k: torch.from_numpy(v) for k, v in host.items()}
        if pin:
            self.host = {k: v.pin_memory() for k, v in self.host.items()}
        self.dev = {k: v.to(device) for k, v in self.host.items()}
        self.D = plan.empty(ARRAY_DIAG, device)
        self.E = plan.empty(ARRAY_OFF, device)
        self.PD = plan.empty(ARRAY_DIAG, device)
        self.PE = plan.empty(ARRAY_OFF, device)
        self.lam = plan.empty(ARRAY_VEC, device)
        n = max(plan.nprob, 1)
        self.iters = torch.zeros(n, dtype=torch.int32, device=device)
        self.relres = torch.zeros(n, dtype=torch.float64, device=device)
        self.status = torch.zeros(n, dtype=torch.int32, device=device)

    def pipeline(self, kind="sym", stream=None):
        d = self.dev
        sspcg_pipeline_batched(self.plan, kind, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], self.D, self.E, self.PD,
                               self.PE, self.lam, self.iters, self.relres, self.status, stream)

    def capture(self, kind, stream):
        d = self.dev
        sspcg_plan_capture_pipeline(self.plan, kind, d["A"], d["B"], d["qd"], d["rd"], d["gamma"], self.D, self.E,
                                    self.PD, self.PE, self.lam, self.iters, self.relres, self.status, stream)

    def lambdas(self) -> List[np.ndarray]:
        return self.plan.unpack(ARRAY_VEC, self.lam, [p.gamma.shape for p in self.probs])
