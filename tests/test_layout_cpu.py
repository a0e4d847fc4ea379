"""Host-side invariants of the PCG shared-memory layout that the host sizing and the kernel share
(pcg_layout, pcg_max_resident), compiled from the library's own header by nvcc and run on the CPU
for every nx, a spread of N and nu, both operator forms and every option that adds vectors:

* every region starts 16-byte aligned (the kernel loads vector segments with 128-bit loads);
* the regions are in order and do not overlap, and the total covers the last one;
* pcg_max_resident returns the largest K whose layout fits (K fits, K + 1 does not), or -1 when
  even the vectors do not fit, and N + 1 when everything fits;
* the global-workspace slot (K = 0) holds the vectors.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_06427_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include "kernels.h"
using namespace sspcg;
static int bad = 0;
static void fail(const char *what, int op, int N, int nx, int nu, int poly, int cg, long long K) {
  if (bad++ < 20) std::printf("FAIL %s op=%d N=%d nx=%d nu=%d poly=%d cg=%d K=%lld\n", what, op, N, nx, nu, poly, cg, K);
}
static void check_layout(int op, int K, int N, int nx, int nu, int poly, int cg) {
  const PcgLayout L = pcg_layout(op, K, N, nx, nu, poly, cg);
  const long long offs[] = {L.p, L.r, L.w, L.x, L.e, L.u, L.s, L.v, L.vu, L.iq, L.ir, L.m0, L.m1, L.pd, L.pe, L.total};
  for (long long o : offs)
    if (o % 4 != 0) fail("alignment", op, N, nx, nu, poly, cg, K);
  // region starts (a vector's region begins one zero segment before its block row 0)
  const long long g = vec_stride(nx);
  const long long starts[] = {L.p - g, L.r - g, L.w - g, L.x - g, L.e - g, L.u - g, L.s - g, L.v - g, L.iq, L.ir,
                              L.m0, L.m1, L.pd, L.pe, L.total};
  for (size_t i = 1; i < sizeof(starts) / sizeof(starts[0]); ++i)
    if (starts[i] < starts[i - 1]) fail("order", op, N, nx, nu, poly, cg, K);
  const long long NXP = vec_stride(nx), RV = (long long)(N + 1) * NXP, RVP = RV + 2 * NXP;
  // every vector has a zero segment before and after it: regions of (N + 3) segments, block row 0 one in
  if (L.p != NXP) fail("front segment", op, N, nx, nu, poly, cg, K);
  // the vectors the kernel always uses are distinct and full length
  const long long vec[] = {L.p, L.r, L.w, L.x};
  for (int i = 1; i < 4; ++i)
    if (vec[i] - vec[i - 1] < RVP) fail("vector overlap", op, N, nx, nu, poly, cg, K);
  if (poly && L.u - L.e < RVP) fail("poly vector", op, N, nx, nu, poly, cg, K);
  if (cg && (L.s - L.u < RVP || L.v - L.s < RVP)) fail("cg vectors", op, N, nx, nu, poly, cg, K);
  if (L.v - L.x < RVP) fail("x vector", op, N, nx, nu, poly, cg, K);
  if (op == kOpQp) {
    const long long NUP = vec_stride(nu);
    // v_x, its back zero segment, v_u's front zero segment, v_u (N rows), then 1/q
    if (L.vu - L.v != RV + NXP + NUP) fail("v_u offset", op, N, nx, nu, poly, cg, K);
    if (L.iq - L.vu < (long long)N * NUP) fail("v_u overlap", op, N, nx, nu, poly, cg, K);
  }
  // a single knot stages one zero off-diagonal slot
  if (N == 0 && K > 0 && L.pd + (long long)nx * pad_ld(nx) > L.pe) fail("pd slot", op, N, nx, nu, poly, cg, K);
  if (N == 0 && K > 0 && L.total - L.pe < (long long)nx * pad_ld(nx)) fail("zero slot", op, N, nx, nu, poly, cg, K);
}
int main() {
  const int Ns[] = {0, 1, 2, 3, 7, 16, 31, 64, 100, 128, 255, 512, 1000};
  for (int op = 0; op <= 1; ++op)
    for (int nx = 1; nx <= kMaxNx; ++nx)
      for (int nu : {0, 1, (nx + 1) / 2, nx})
        for (int N : Ns)
          for (int poly = 0; poly <= 1; ++poly)
            for (int cg = 0; cg <= 1; ++cg) {
              if (cg && op != kOpQp) continue;
              for (int K : {0, 1, N / 2, N, N + 1}) check_layout(op, K, N, nx, nu, poly, cg);
              for (long long elems : {1000LL, 20000LL, 56000LL, 1LL << 20}) {
                const int K = pcg_max_resident(op, N, nx, nu, elems, poly, cg);
                if (K == -1) {
                  if (pcg_layout(op, 0, N, nx, nu, poly, cg).total <= elems) fail("fits at K=0", op, N, nx, nu, poly, cg, K);
                  continue;
                }
                if (K < 0 || K > N + 1) fail("range", op, N, nx, nu, poly, cg, K);
                if (pcg_layout(op, K, N, nx, nu, poly, cg).total > elems) fail("K does not fit", op, N, nx, nu, poly, cg, K);
                if (K <= N && pcg_layout(op, K + 1, N, nx, nu, poly, cg).total <= elems)
                  fail("K not maximal", op, N, nx, nu, poly, cg, K);
              }
            }
  std::printf(bad ? "%d failures\n" : "ok\n", bad);
  return bad ? 1 : 0;
}
'''


def test_layout_invariants(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "layout_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", f"-I{CSRC}", str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
