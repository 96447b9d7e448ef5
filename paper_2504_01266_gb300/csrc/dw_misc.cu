// dw_misc.cu -- the two small kernels around the depthwise backward pass:
//  * the clamp-border edge fold of the input gradient, and
//  * the FP64 fixed-order reduction of the per-CTA filter-gradient partials.
#include <algorithm>

#include "dw_fold.cuh"
#include "dw_kernels.cuh"
#include "dw_launch.h"

namespace giga {

int64_t dw_bwd_chunks_per_plane(int64_t H, int64_t W, int tiles_per_cta) {
  const int64_t tiles = ((W + kTileW - 1) / kTileW) * ((H + kBwdTileH - 1) / kBwdTileH);
  return (tiles + tiles_per_cta - 1) / tiles_per_cta;
}

// ------------------------------------------------------------- edge fold
template <typename T>
__global__ void dw_fixup_kernel(const T* __restrict__ dy, const float* __restrict__ w,
                                T* __restrict__ dx, int C, int H, int W, int K,
                                int64_t edge_per_plane, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t plane = e / edge_per_plane;
    const int64_t k = e - plane * edge_per_plane;
    fold_edge_pixel<T>(dy + plane * (int64_t)H * W, w + (int64_t)(plane % C) * K * K,
                       dx + plane * (int64_t)H * W, H, W, K, k);
  }
}

cudaError_t dw_fixup_launch(const DwArgs& a, cudaStream_t st) {
  if (a.border != 1 || a.N * a.C * a.H * a.W == 0) return cudaSuccess;
  const int64_t H = a.H, W = a.W;
  const int64_t edge = edge_pixels(H, W);
  const int64_t total = a.N * a.C * edge;
  const int threads = 128;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 65535);
  if (a.dtype == 0)
    dw_fixup_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const float*>(a.dy), a.w, static_cast<float*>(a.dx), (int)a.C, (int)H,
        (int)W, a.K, edge, total);
  else
    dw_fixup_kernel<__nv_bfloat16><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const __nv_bfloat16*>(a.dy), a.w, static_cast<__nv_bfloat16*>(a.dx),
        (int)a.C, (int)H, (int)W, a.K, edge, total);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------ FP64 reduction
// One warp per (channel, tap): lanes stride over the (image, chunk) partials
// in a fixed order, accumulate in FP64 and combine with a fixed butterfly, so
// the result does not depend on scheduling.
__global__ void dw_finalize_kernel(const float* __restrict__ partials, float* __restrict__ dw,
                                   int64_t N, int C, int64_t chunks, int KK) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)C * KK) return;
  const int c = (int)(gw / KK), k = (int)(gw % KK);
  double s = 0.0;
  const int64_t count = N * chunks;
  for (int64_t idx = lane; idx < count; idx += 32) {
    const int64_t n = idx / chunks, ch = idx - n * chunks;
    s += (double)partials[((n * C + c) * chunks + ch) * KK + k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) dw[(int64_t)c * KK + k] = (float)s;
}

cudaError_t dw_finalize_launch(const DwArgs& a, int64_t chunks_per_plane, cudaStream_t st) {
  const int KK = a.K * a.K;
  const int64_t warps = a.C * KK;
  const int threads = 256;
  const int64_t blocks = (warps * 32 + threads - 1) / threads;
  dw_finalize_kernel<<<(unsigned)blocks, threads, 0, st>>>(a.partials, a.dw, a.N, (int)a.C,
                                                           chunks_per_plane, KK);
  note_launch();
  return cudaGetLastError();
}

}  // namespace giga
