// peak.cu -- FP32 fused multiply-add throughput of the device, measured.
//
// The depthwise kernels with K >= 7 are bound by FP32 FMA issue, not by HBM,
// so their roofline needs the FMA rate this GPU actually sustains.  Counting
// units (SMs x FP32 lanes x clock) assumes the SM count and the clock; this
// kernel measures the rate instead: every thread runs 16 independent
// multiply-add chains (enough to cover the FMA latency with 8 warps per
// scheduler), in plain `fma.rn.f32` form or in the packed `fma.rn.f32x2`
// form (two FP32 FMAs per instruction), over all SMs.  The values stay finite
// (a contraction towards c / (1 - m)); the sums are stored so the chains are
// not dead code.  Not part of the paper's method: measurement support.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace giga {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;
constexpr int kPeakChains = 16;

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* __restrict__ sink,
                                                                int iters, float m, float c) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const float seed = (float)(tid & 255) * 1e-3f;
  float total = 0.f;
  if constexpr (!PACKED) {
    float acc[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) acc[i] = seed + (float)i;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int rep = 0; rep < 4; ++rep)
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i)
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[i]) : "f"(m), "f"(c));
    }
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) total += acc[i];
  } else {
    uint64_t acc[kPeakChains / 2];
    const uint64_t m2 = pack2(m, m), c2 = pack2(c, c);
#pragma unroll
    for (int i = 0; i < kPeakChains / 2; ++i) acc[i] = pack2(seed + 2 * i, seed + 2 * i + 1);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int rep = 0; rep < 4; ++rep)
#pragma unroll
        for (int i = 0; i < kPeakChains / 2; ++i)
          asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[i]) : "l"(m2), "l"(c2));
    }
#pragma unroll
    for (int i = 0; i < kPeakChains / 2; ++i)
      total += __uint_as_float((uint32_t)acc[i]) + __uint_as_float((uint32_t)(acc[i] >> 32));
  }
  sink[tid] = total;
}

}  // namespace giga

using namespace giga;

extern "C" size_t giga_fp32_fma_peak_sink_bytes(void) {
  return sizeof(float) * (size_t)sm_count() * kPeakBlocksPerSm * kPeakThreads;
}

extern "C" giga_status_t giga_fp32_fma_peak(int32_t packed, float* sink, size_t sink_bytes,
                                            double* tflops, double* ms, void* stream) {
  clear_error();
  if (!tflops) return fail(GIGA_ERR_INVALID_ARG, "tflops is NULL");
  *tflops = 0.0;
  if (ms) *ms = 0.0;
  if (packed != 0 && packed != 1) return fail(GIGA_ERR_INVALID_ARG, "packed must be 0 or 1");
  const int blocks = sm_count() * kPeakBlocksPerSm;
  const size_t need = sizeof(float) * (size_t)blocks * kPeakThreads;
  if (!sink || sink_bytes < need)
    return fail(GIGA_ERR_WORKSPACE, "sink must hold giga_fp32_fma_peak_sink_bytes() bytes");
  if (reinterpret_cast<uintptr_t>(sink) % 4) return fail(GIGA_ERR_MISALIGNED, "sink");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // 16 chains x 4 repeats x 2 FLOP per iteration and thread: ~4 ms per launch
  // at 80 TFLOP/s on 152 SMs
  const int iters = 20000;
  auto launch = [&]() {
    if (packed)
      fma_peak_kernel<true><<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
    else
      fma_peak_kernel<false><<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
    note_launch();
    return cudaGetLastError();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();  // warm-up (clocks up, code loaded)
  float best = 1e30f;
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) best = std::min(best, t);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "FMA throughput kernel");
  const double flop = 2.0 * kPeakChains * 4 * (double)iters * blocks * kPeakThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return GIGA_OK;
}
