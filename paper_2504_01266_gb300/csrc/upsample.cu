// upsample.cu -- nearest-neighbour upsampling by an integer factor s (the
// GigaAPI paper, Section 4.2.3) and the paper's sharpening benchmark fused
// into one pass (Section 6.6): the K x K depthwise filter applied to the
// upsampled image without storing it.  K = 3 (the paper's Laplacian) runs the
// polyphase kernel, which applies the taps summed per input pixel to the input
// directly; larger K run the tile kernel, which expands the staged input rows
// in shared memory and filters them.
//
//   up[n][c][p][q] = x[n][c][p / s][q / s]                      (integer division)
//   y[n][c][p][q]  = sum_{a,b} w[c][a][b] * up~[n][c][p + a - r][q + b - r]
//
// up~ applies the border rule on the (H*s) x (W*s) upsampled image.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dw_launch.h"
#include "upsample.cuh"

namespace giga {

// --------------------------------------------------------------- upsample
// One thread per 4 consecutive outputs of a row (a 16/8-byte store when the
// row allows it).  The chunk index splits into (row, chunk of row) by a
// fixed-divisor division; the 4 source columns follow q0 / s incrementally.
template <typename T>
__global__ void __launch_bounds__(256) up_nearest_kernel(const T* __restrict__ x,
                                                         T* __restrict__ y, int H, int W,
                                                         int Ho, int Wo, FastDiv fs,
                                                         FastDiv fcpr, FastDiv fho,
                                                         uint32_t chunks, int vec) {
  const uint32_t cpr = fcpr.d;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < chunks;
       k += gridDim.x * blockDim.x) {
    const uint32_t row = fdiv(k, fcpr);  // plane * Ho + p
    const int q0 = (int)(k - row * cpr) * 4;
    const uint32_t plane = fdiv(row, fho);
    const int p = (int)(row - plane * (uint32_t)Ho);
    const T* src = x + ((int64_t)plane * H + fdiv((uint32_t)p, fs)) * (int64_t)W;
    T* dst = y + (int64_t)row * Wo + q0;
    int sv = (int)fdiv((uint32_t)q0, fs), rem = q0 - sv * fs.d;
    float e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      e[q] = q0 + q < Wo ? Elem<T>::load(src + sv) : 0.f;
      if (++rem == (int)fs.d) {
        rem = 0;
        ++sv;
      }
    }
    if (vec && q0 + 3 < Wo) {
      Elem<T>::store4(dst, make_float4(e[0], e[1], e[2], e[3]));
    } else {
      for (int q = 0; q < 4 && q0 + q < Wo; ++q) Elem<T>::store(dst + q, e[q]);
    }
  }
}

// Persistent warps, each on its own sequence of items (plane, group of
// kUp3Rows input rows, block of 32 PX input columns; the column block fastest),
// the summed taps recomputed when the channel changes.
constexpr int kUp3Warps = 8;

template <typename T, int CE, int S, int PX>
__global__ void __launch_bounds__(kUp3Warps * 32) up3_poly_kernel(
    const T* __restrict__ x, const float* __restrict__ w, T* __restrict__ y, FastDiv fc, int H,
    int W, int s, FastDiv fcb, FastDiv frb, uint32_t items, int clamp) {
  if (S) s = S;
  float wt[36];
  int c_cur = -1;
  for (uint32_t item = blockIdx.x * kUp3Warps + (threadIdx.x >> 5); item < items;
       item += gridDim.x * kUp3Warps) {
    const uint32_t q = fdiv(item, fcb);
    const int cb = (int)(item - q * fcb.d);
    const uint32_t plane = fdiv(q, frb);
    const int rg = (int)(q - plane * frb.d);
    const int c = (int)(plane - fdiv(plane, fc) * fc.d);
    if (c != c_cur) {
      up3_weights<S>(w + (int64_t)c * 9, wt);
      c_cur = c;
    }
    up3_item<T, CE, S, PX>(x + (int64_t)plane * H * W,
                           y + (int64_t)plane * H * s * ((int64_t)W * s), H, W, s, rg * kUp3Rows,
                           cb, clamp, wt);
  }
}

// ------------------------------------------------- upsample, then filter
// One 64 x 128 output tile of the upsampled grid at a time per CTA (8 warps,
// 8 rows each), over tiles t = blockIdx.x, + gridDim.x, ... (launched with one
// tile per CTA: measured faster than persistent CTAs, which need a second
// stage); scale s >= 2 (scale 1 is the plain forward).  Per tile: the input pixels
// its halo window needs (rows and columns of the upsampled window divided by
// s, clamped to the image) and its plane's filter are copied to one of two
// stages -- those of the next tile are copied while this one is computed --
// then up_tile expands them along the columns and filters the tile.
template <typename T, int K>
__device__ __forceinline__ void up_fwd_body(const T* __restrict__ x, const float* __restrict__ w,
                                            T* __restrict__ y, FastDiv fc, int H, int W, int Ho,
                                            int Wo, FastDiv fs, FastDiv ftx, FastDiv fty,
                                            int64_t num_tiles, int clamp, int vec) {
  using G = Geo<K>;
  using U = UpShape<K>;
  extern __shared__ __align__(16) float smem[];
  float* sx = smem;                                  // expanded input rows + a zero row
  int* scol = reinterpret_cast<int*>(sx + U::EXP);   // SP column map
  int* rowoff = scol + G::SP;                        // ROWS: offset of each halo row in sx
  // 1 or 2 x {filter, SRC_ROWS x SRC_COLS pixels}; the second only when a CTA
  // runs several tiles
  float* stages = reinterpret_cast<float*>(scol) + U::TABLES;

  struct Tile {
    int ty0, tx0, su0, sv0, nr, nc;
    int plane;
  };
  auto locate = [&](int64_t t) {  // t < 2^31
    Tile tl;
    const uint32_t u = (uint32_t)t;
    const uint32_t t2 = fdiv(u, ftx);
    tl.tx0 = (int)(u - t2 * ftx.d) * kTileW;
    const uint32_t pl = fdiv(t2, fty);
    tl.ty0 = (int)(t2 - pl * fty.d) * U::TH;
    tl.plane = (int)pl;
    // input window: upsampled rows [ty0 - r, ty0 + TH + r), columns
    // [tx0 - RP, tx0 + 128 + RP), clamped to the upsampled image, divided by s
    const int u_lo = max(tl.ty0 - G::R, 0), u_hi = min(tl.ty0 + U::TH + G::R, Ho) - 1;
    const int v_lo = max(tl.tx0 - G::RP, 0), v_hi = min(tl.tx0 + kTileW + G::RP, Wo) - 1;
    tl.su0 = (int)fdiv((uint32_t)u_lo, fs);
    tl.sv0 = (int)fdiv((uint32_t)v_lo, fs);
    tl.nr = (int)fdiv((uint32_t)u_hi, fs) - tl.su0 + 1;  // <= SRC_ROWS
    tl.nc = (int)fdiv((uint32_t)v_hi, fs) - tl.sv0 + 1;  // <= SRC_COLS
    return tl;
  };
  // copy tile tl's filter and input pixels to stage b, every copy in flight
  // at once (FP32: 4-byte cp.async; BF16: loads issued before the widened
  // stores); one commit group per stage
  auto stage = [&](const Tile& tl, int b) {
    float* sw = stages + b * U::STAGE;
    float* ss = sw + round_up(G::WPAD, 4);
    const int c = tl.plane - (int)(fdiv((uint32_t)tl.plane, fc) * fc.d);
    stage_filter_async<K>(sw, w + (int64_t)c * K * K, false, kThreads);
    const T* xp = x + (int64_t)tl.plane * H * W + (int64_t)tl.su0 * W + tl.sv0;
    up_stage_pixels<T, U::SRC_ROWS * U::SRC_COLS>(ss, U::SRC_COLS, xp, W, tl.nr, tl.nc);
    cp_async_commit();
  };

  int64_t t = blockIdx.x;
  if (t >= num_tiles) return;
  Tile cur = locate(t);
  stage(cur, 0);
  for (int k = threadIdx.x; k < G::SP; k += kThreads) sx[U::ZERO_OFF + k] = 0.f;
  for (int b = 0; t < num_tiles; t += gridDim.x, b ^= 1) {
    const int64_t tn = t + gridDim.x;
    Tile nxt;
    if (tn < num_tiles) {
      nxt = locate(tn);
      stage(nxt, b ^ 1);  // that stage was last read before the previous tile's barriers
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    const float* sw = stages + b * U::STAGE;
    const float* ss = sw + round_up(G::WPAD, 4);
    up_tile<T, K>(sx, U::ZERO_OFF, scol, rowoff, sw, ss, U::SRC_COLS, cur.ty0, cur.tx0, cur.su0,
                  cur.sv0, cur.nr, Ho, Wo, fs, clamp != 0, y + (int64_t)cur.plane * Ho * Wo,
                  vec != 0);
    cur = nxt;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) up_fwd_kernel(const T* __restrict__ x,
                                                          const float* __restrict__ w,
                                                          T* __restrict__ y, FastDiv fc, int H,
                                                          int W, int Ho, int Wo, FastDiv fs,
                                                          FastDiv ftx, FastDiv fty,
                                                          int64_t num_tiles, int clamp, int vec) {
  up_fwd_body<T, K>(x, w, y, fc, H, W, Ho, Wo, fs, ftx, fty, num_tiles, clamp, vec);
}

// The kernel of a launch; raises its shared-memory limit first.
template <typename T, int K>
static cudaError_t up_kernel_for(size_t smem, decltype(&up_fwd_kernel<T, K>)* kern) {
  *kern = up_fwd_kernel<T, K>;
  return set_smem_once<up_fwd_kernel<T, K>>(smem);
}

template <typename T, int K>
static cudaError_t up_fwd_impl(const UpArgs& a, cudaStream_t st) {
  using U = UpShape<K>;
  const size_t smem = (size_t)U::SM_FLOATS * 4;
  decltype(&up_fwd_kernel<T, K>) kern = nullptr;
  cudaError_t e = up_kernel_for<T, K>(smem, &kern);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.Wo + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.Ho + U::TH - 1) / U::TH;
  const int64_t tiles = a.N * a.C * tiles_x * tiles_y;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int64_t grid = tiles;  // one tile per CTA: the second stage is never used
  const size_t smem1 = (size_t)U::SM_FLOATS_1 * 4;
  kern<<<(unsigned)grid, kThreads, smem1, st>>>(
      static_cast<const T*>(a.x), a.w, static_cast<T*>(a.y), make_fastdiv((uint32_t)a.C),
      (int)a.H, (int)a.W, (int)a.Ho, (int)a.Wo, make_fastdiv((uint32_t)a.s),
      make_fastdiv((uint32_t)tiles_x), make_fastdiv((uint32_t)tiles_y), tiles, a.border, a.vec);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int CE, int S, int PX>
static cudaError_t up3_launch_ce(const UpArgs& a, cudaStream_t st) {
  const int64_t rgs = (a.H + kUp3Rows - 1) / kUp3Rows;
  const int64_t cbs = (a.W + 32 * PX - 1) / (32 * PX);
  const int64_t items = a.N * a.C * rgs * cbs;
  if (items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  static int ctas_per_sm[64] = {};  // per device, measured at its first launch
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, up3_poly_kernel<T, CE, S, PX>, kUp3Warps * 32, 0);
    if (e != cudaSuccess) return e;
    per_sm = n > 0 ? n : 1;
  }
  const int64_t grid = std::min<int64_t>((items + kUp3Warps - 1) / kUp3Warps,
                                         (int64_t)per_sm * sm_count());
  up3_poly_kernel<T, CE, S, PX><<<(unsigned)grid, kUp3Warps * 32, 0, st>>>(
      static_cast<const T*>(a.x), a.w, static_cast<T*>(a.y), make_fastdiv((uint32_t)a.C),
      (int)a.H, (int)a.W, a.s, make_fastdiv((uint32_t)cbs), make_fastdiv((uint32_t)rgs),
      (uint32_t)items, a.border);
  note_launch();
  return cudaGetLastError();
}

// K = 3: the polyphase kernel compiled for the mode up3_mode picks.
template <typename T>
static cudaError_t up3_launch(const UpArgs& a, cudaStream_t st) {
  constexpr int kSector = 32 / (int)sizeof(T);
  switch (up3_mode(a.s, a.y, (int)sizeof(T), a.W)) {
    case 0: return up3_launch_ce<T, 4, 2, 2>(a, st);
    case 1: return up3_launch_ce<T, 8, 4, 2>(a, st);
    case 2: return up3_launch_ce<T, 2, 2, 1>(a, st);
    case 3: return up3_launch_ce<T, 4, 4, 1>(a, st);
    case 4: return up3_launch_ce<T, 8, 8, 1>(a, st);
    case 5: return up3_launch_ce<T, kSector, 0, 1>(a, st);
    case 6:
      if constexpr (sizeof(T) == 2) return up3_launch_ce<T, 8, 0, 1>(a, st);
      return cudaErrorInvalidValue;
    case 7: return up3_launch_ce<T, 4, 0, 1>(a, st);
    case 8: return up3_launch_ce<T, 2, 0, 1>(a, st);
    default: return up3_launch_ce<T, 1, 0, 1>(a, st);
  }
}

template <typename T>
static cudaError_t up_fwd_dispatch(const UpArgs& a, cudaStream_t st) {
  switch (a.K) {
    case 1: return up_fwd_impl<T, 1>(a, st);
    case 3: return up3_launch<T>(a, st);
    case 5: return up_fwd_impl<T, 5>(a, st);
    case 7: return up_fwd_impl<T, 7>(a, st);
    case 9: return up_fwd_impl<T, 9>(a, st);
    case 11: return up_fwd_impl<T, 11>(a, st);
    case 13: return up_fwd_impl<T, 13>(a, st);
    case 15: return up_fwd_impl<T, 15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t up_fwd_launch(const UpArgs& a, cudaStream_t st) {
  return a.dtype == 0 ? up_fwd_dispatch<float>(a, st) : up_fwd_dispatch<__nv_bfloat16>(a, st);
}

cudaError_t up_nearest_launch(const UpArgs& a, cudaStream_t st) {
  const int64_t cpr = (a.Wo + 3) / 4;
  const int64_t chunks = a.N * a.C * a.Ho * cpr;
  if (chunks >= (1LL << 32) || a.N * a.C * a.Ho >= (1LL << 32)) return cudaErrorInvalidValue;
  const int64_t want = (chunks + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count() * 16);
  const FastDiv fs = make_fastdiv((uint32_t)a.s), fc = make_fastdiv((uint32_t)cpr),
                fh = make_fastdiv((uint32_t)a.Ho);
  if (a.dtype == 0)
    up_nearest_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(a.x),
                                                   static_cast<float*>(a.y), (int)a.H, (int)a.W,
                                                   (int)a.Ho, (int)a.Wo, fs, fc, fh,
                                                   (uint32_t)chunks, a.vec);
  else
    up_nearest_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
        static_cast<const __nv_bfloat16*>(a.x), static_cast<__nv_bfloat16*>(a.y), (int)a.H,
        (int)a.W, (int)a.Ho, (int)a.Wo, fs, fc, fh, (uint32_t)chunks, a.vec);
  note_launch();
  return cudaGetLastError();
}

}  // namespace giga
