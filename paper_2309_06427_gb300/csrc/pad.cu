// Padded copies of the block rows that the PCG kernel streams from global
// memory.  A problem that does not fit in shared memory whole reads its
// remaining block rows of A, B and PE every iteration, row-wise as well as
// column-wise.  In the packed input layout a row of A_k starts at a multiple
// of nx values, so for odd nx the row-wise reads cannot use 128-bit loads.
// Each warp load then touches 32 sectors, and the L1 looks each sector up
// once for every column it holds.  These copies give every row nx (or nu)
// rounded up to 4 values, zero-padded, so the kernel reads a row 16 bytes at
// a time.  The PCG reads the streamed rows from the copies only, in both
// orientations, so the L2 working set grows only by the padding.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace sspcg {
namespace {

constexpr int kPadThreads = 256;

// rows of width w (dense, src) into rows of width wp >= w, wp a multiple of 4 (dst), zeros past w.  The CTA's
// threads each write 16 bytes per step: piece v is values 4 c .. 4 c + 3 of padded row r (a piece never
// crosses rows), r = v / (wp / 4) in FP32, exact for v < 2^20 (at most 4096 x 28 rows of 7 pieces).
__device__ __forceinline__ void pad_block_rows(float *dst, const float *src, int rows, int w, int wp) {
  const int q4 = wp >> 2;
  const float inv_q4 = 1.0f / (float)q4;
  const int n = rows * q4;
  float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll 4
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int r = (int)(((float)v + 0.5f) * inv_q4);
    const int c = 4 * (v - r * q4);
    const float *s = src + (int64_t)r * w;
    float4 o;
    o.x = c < w ? __ldg(s + c) : 0.0f;
    o.y = c + 1 < w ? __ldg(s + c + 1) : 0.0f;
    o.z = c + 2 < w ? __ldg(s + c + 2) : 0.0f;
    o.w = c + 3 < w ? __ldg(s + c + 3) : 0.0f;
    d4[v] = o;
  }
}

// One CTA per listed problem (grid-stride).
__global__ void __launch_bounds__(kPadThreads) pad_rows_kernel(const ProbDesc *desc, const int32_t *list,
                                                               int32_t count, const float *A, const float *B,
                                                               const float *PE, const int64_t *pad_off,
                                                               float *pad) {
  for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
    const ProbDesc d = desc[list[q]];
    const int64_t po = pad_off[d.id];
    if (po < 0 || d.N == 0) continue;
    const int nxp = vec_stride(d.nx), nup = vec_stride(d.nu);
    const int rows = d.N * d.nx;
    pad_block_rows(pad + po, A + d.oA, rows, d.nx, nxp);
    const int64_t ra = pad_region(rows, d.nx), rb = pad_region(rows, d.nu);
    if (d.nu > 0) pad_block_rows(pad + po + ra, B + d.oB, rows, d.nu, nup);
    if (PE) pad_block_rows(pad + po + ra + rb, PE + d.ooff, rows, d.nx, nxp);
  }
}

}  // namespace

cudaError_t launch_pad_rows(const ProbDesc *desc, const int32_t *list, int32_t count, const float *A,
                            const float *B, const float *PE, const int64_t *pad_off, float *pad, int sms,
                            cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>(count, (int64_t)8 * sms);
  pad_rows_kernel<<<grid, kPadThreads, 0, st>>>(desc, list, count, A, B, PE, pad_off, pad);
  return cudaGetLastError();
}

}  // namespace sspcg
