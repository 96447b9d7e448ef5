// common.cuh -- shared definitions of the libgiga CUDA sources (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace giga {

// Tile geometry of the depthwise kernels: a CTA of 8 warps owns a tile of
// TILE_H x TILE_W output pixels of one image plane; each lane owns 4
// consecutive columns, so one warp row spans 128 columns and every global
// access of a warp row is one contiguous 512-byte (FP32) segment.
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTileW = 128;

// Unsigned division by a fixed divisor d >= 1 as a multiply-high and a shift:
// with 2^(l-1) < d <= 2^l, mul = ceil(2^(31+l) / d) < 2^32 exceeds 2^(31+l) / d
// by e / d, e < d <= 2^l, so n * e < 2^(31+l) and the quotient is exact for
// every n < 2^31.  Tile and plane indices are split this way instead of by
// 64-bit division, which the compiler emulates with a long instruction
// sequence.
struct FastDiv {
  uint32_t mul, shift, d;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{0, 0, d};
  if (d <= 1) {
    f.d = 1;
    return f;
  }
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.shift = l - 1;
  f.mul = (uint32_t)((((uint64_t)1 << (32 + f.shift)) + d - 1) / d);
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return f.d == 1 ? n : (__umulhi(n, f.mul) >> f.shift);
}

// Depthwise problem as seen by the launchers (all pointers device memory).
struct DwArgs {
  const void* x;
  const void* dy;
  const float* w;
  void* y;
  void* dx;
  float* dw;
  float* partials;  // workspace: per-CTA FP32 filter-gradient partial sums
  int64_t N, C, H, W;
  int K;
  int border;  // 0 zero, 1 clamp
  int dtype;   // 0 f32, 1 bf16
  int vec;     // 1: every row starts 16 B (f32) / 8 B (bf16) aligned
};

// Launch configuration chosen by the autotuner (or the defaults).
struct DwConfig {
  int rows_per_thread;  // forward / input-gradient kernel: 4 or 8
  int persistent;       // forward / input-gradient kernel: 1 = persistent, double-buffered
  int prefetch;         // forward / input-gradient kernel: 1 = L2 prefetch of a later tile
  int tiles_per_cta;    // filter-gradient kernels: consecutive tiles per chunk
  int split;            // fused backward: 1 = input and filter gradients as two passes
  int ring;             // fused backward: 1 = persistent kernel with a two-stage tile ring
};

// Element access for the two storage types; arithmetic is always FP32.
template <typename T> struct Elem;
template <> struct Elem<float> {
  static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float4 load4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
  static __device__ __forceinline__ void store4(float* p, float4 v) {
    *reinterpret_cast<float4*>(p) = v;
  }
};
template <> struct Elem<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    float4 f;
    f.x = __uint_as_float(u.x << 16);
    f.y = __uint_as_float(u.x & 0xffff0000u);
    f.z = __uint_as_float(u.y << 16);
    f.w = __uint_as_float(u.y & 0xffff0000u);
    return f;
  }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ void store4(__nv_bfloat16* p, float4 v) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(p) = u;
  }
};

// Host-side launch accounting (giga_launch_count).
void note_launch(int n = 1);

// Multiprocessors of the current device (cached per device).
int sm_count();

// Raise a kernel's dynamic shared-memory limit once per device (the attribute
// is per context; later calls are a bit test).  One flag word per kernel.
template <auto kern>
inline cudaError_t set_smem_once(size_t bytes) {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace giga
