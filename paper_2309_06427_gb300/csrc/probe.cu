// Shared-memory read bandwidth of this GPU, measured: the peak the PCG
// kernel's roofline is reported against.  Every thread reads a 48 KB
// shared-memory buffer with conflict-free 32-bit or 128-bit loads (warp w
// reads 32 consecutive words or 16-byte words per load) and sums what it
// reads; two 1024-thread CTAs per SM; the sums go to a small device buffer
// so the loads cannot be dropped.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sspcg.h"
#include "common.cuh"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeBytes = 48 * 1024;

// Loads that neither the compiler nor ptxas may drop or hoist out of the rounds loop: ld.volatile in the
// PTX itself (a volatile asm statement alone still emits a plain ld.shared, which ptxas may hoist).
template <int B>
__device__ __forceinline__ float lds(uint32_t addr);
template <>
__device__ __forceinline__ float lds<4>(uint32_t addr) {
  float v;
  asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
template <>
__device__ __forceinline__ float lds<16>(uint32_t addr) {
  float a, b, c, d;
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a), "=f"(b), "=f"(c), "=f"(d) : "r"(addr));
  return (a + b) + (c + d);
}

template <int B>
__global__ void __launch_bounds__(kProbeThreads, 2) smem_read_kernel(int rounds, float *sink) {
  constexpr int per = kProbeBytes / (kProbeThreads * B);  // loads per thread per round
  __shared__ __align__(16) float buf[kProbeBytes / 4];
  for (int e = threadIdx.x; e < kProbeBytes / 4; e += kProbeThreads) buf[e] = (float)(e & 7);
  __syncthreads();
  // thread t reads word (or 16-byte word) t + k * 1024: a warp reads one contiguous run per load
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf) + threadIdx.x * B;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < per; ++k) acc[k & 3] += lds<B>(base + k * kProbeThreads * B);
  }
  sink[blockIdx.x * kProbeThreads + threadIdx.x] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

}  // namespace

extern "C" sspcg_status sspcg_measure_smem_bandwidth(int32_t load_bytes, int32_t rounds, double *gbytes_per_s,
                                                     sspcg_stream stream) {
  if (!gbytes_per_s || rounds <= 0 || (load_bytes != 4 && load_bytes != 16)) return SSPCG_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SSPCG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SSPCG_ERR_CUDA;
  const int grid = 2 * sms;
  cudaStream_t st = (cudaStream_t)stream;
  float *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * grid * kProbeThreads) != cudaSuccess) return SSPCG_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int r) {
    if (load_bytes == 16) smem_read_kernel<16><<<grid, kProbeThreads, 0, st>>>(r, sink);
    else smem_read_kernel<4><<<grid, kProbeThreads, 0, st>>>(r, sink);
  };
  launch(rounds / 4 + 1);  // warm-up (clocks, module load)
  cudaEventRecord(e0, st);
  launch(rounds);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || ms <= 0.0f) return SSPCG_ERR_CUDA;
  *gbytes_per_s = (double)grid * kProbeThreads * (double)rounds * (kProbeBytes / kProbeThreads) / (ms * 1e-3) / 1e9;
  return SSPCG_OK;
}
