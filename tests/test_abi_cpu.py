"""CPU checks of the C-ABI library: it builds, loads, exports every symbol the
header declares, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sspcg.h")


@pytest.fixture(scope="module")
def L():
    from paper_2309_06427_gb300 import build
    build.build()
    from paper_2309_06427_gb300 import sspcg
    return sspcg.lib()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sspcg_status|const char \*)\s*(sspcg_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("sspcg_build_schur", "sspcg_build_precond", "sspcg_solve", "sspcg_solve_qp",
                 "sspcg_build_schur_batched", "sspcg_build_precond_batched", "sspcg_solve_batched",
                 "sspcg_plan_create", "sspcg_plan_destroy", "sspcg_pipeline_host"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert b"sm_103a" in L.sspcg_version()


def test_invalid_shapes_rejected_on_host(L):
    from paper_2309_06427_gb300 import sspcg
    o = sspcg.options()
    vp = ctypes.c_void_p(16)
    # nx out of range, N negative, nu out of range: rejected before any CUDA call
    assert L.sspcg_build_schur(4, 29, 2, vp, vp, vp, vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    assert L.sspcg_build_schur(-1, 4, 2, vp, vp, vp, vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    assert L.sspcg_build_schur(4, 4, 29, vp, vp, vp, vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    assert L.sspcg_build_precond(4, 4, 9, vp, vp, vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    # null outputs
    assert L.sspcg_build_schur(4, 4, 2, vp, vp, vp, vp, None, vp, None) == sspcg.ERR_INVALID_ARG
    assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, None, ctypes.byref(o), vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    # bad options
    bad = sspcg.options(block_threads=33)
    assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, vp, ctypes.byref(bad), vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    bad = sspcg.options(tol=-1.0)
    assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, vp, ctypes.byref(bad), vp, vp, vp, None) == sspcg.ERR_INVALID_ARG
    for deg in (-1, sspcg.MAX_POLY_DEGREE + 1):
        bad = sspcg.options(poly_degree=deg)
        assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, vp, ctypes.byref(bad), vp, vp, vp, None) == \
            sspcg.ERR_INVALID_ARG
    # schedules: auto, resident, stream, warp (one problem per warp); anything else is rejected
    assert sspcg.SCHED == {"auto": 0, "resident": 1, "stream": 2, "warp": 3}
    for sched in (-1, 4):
        bad = sspcg.options()
        bad.schedule = sched
        assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, vp, ctypes.byref(bad), vp, vp, vp, None) == \
            sspcg.ERR_INVALID_ARG
    # single-reduction PCG: variant 0 or 1, double-float sums (polynomial preconditioners are allowed)
    for bad in (sspcg.options(cg_variant=2), sspcg.options(cg_variant=1, reduction="f32")):
        assert L.sspcg_solve(4, 4, vp, vp, vp, vp, vp, vp, ctypes.byref(bad), vp, vp, vp, None) == \
            sspcg.ERR_INVALID_ARG
    # plan with a bad shape
    import numpy as np
    h = ctypes.c_void_p()
    N = np.array([3, 4], np.int32); nx = np.array([2, 40], np.int32); nu = np.array([1, 1], np.int32)
    assert L.sspcg_plan_create(ctypes.byref(h), 2, N.ctypes.data, nx.ctypes.data, nu.ctypes.data,
                               ctypes.byref(o)) == sspcg.ERR_INVALID_ARG
    assert L.sspcg_plan_destroy(None) == sspcg.ERR_INVALID_ARG


def test_full_cost_work_size_on_host(L):
    from paper_2309_06427_gb300 import sspcg
    out = ctypes.c_int64(-1)
    # (N+1) nx^2 rounded up to 4, then N nu^2: 5 * 9 -> 48, + 4 * 4
    assert L.sspcg_schur_full_work_floats(4, 3, 2, ctypes.byref(out)) == sspcg.OK and out.value == 64
    assert L.sspcg_schur_full_work_floats(4, 29, 2, ctypes.byref(out)) == sspcg.ERR_INVALID_ARG
    vp = ctypes.c_void_p(16)
    # missing work buffer: rejected before any CUDA call
    assert L.sspcg_build_schur_full(4, 3, 2, vp, vp, vp, vp, vp, vp, None, vp, None) == sspcg.ERR_INVALID_ARG


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2309_06427_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "sspcg_oracle" not in txt and "liboracle" not in txt, f


def _declared_arity():
    """Parameter count of every function the header declares (comments removed, depth-0 commas)."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:sspcg_status|const char \*)\s*(sspcg_\w+)\s*\(([^;]*?)\)\s*;", txt, re.M | re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header(L):
    """Every ctypes signature the binding sets has the header's parameter count (a wrong count passes
    garbage for the trailing arguments)."""
    arity = _declared_arity()
    assert len(arity) >= 40
    checked = 0
    for name, n in arity.items():
        f = getattr(L, name)
        if f.argtypes is not None:
            assert len(f.argtypes) == n, (name, len(f.argtypes), n)
            checked += 1
    assert checked >= 40
