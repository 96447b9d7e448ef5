// dw_kernels.cuh -- depthwise K x K filtering kernels (forward, input
// gradient, filter gradient) for sm_103a.
//
// Operation (GigaAPI paper, Section 4.2.4 "Sharpening", widened to odd K,
// depthwise channels, zero/clamp borders and both gradients):
//   y[n][c][i][j]  = sum_{a,b} w[c][a][b] * x~[n][c][i + a - r][j + b - r]
//   g[n][c][u][v]  = sum_{a,b} w[c][K-1-a][K-1-b] * dy~[n][c][u + a - r][v + b - r]
//                    (dy~ zero outside the image; dx = g for the zero border,
//                    the clamp border adds the edge fold of dw_fixup.cu)
//   dw[c][a][b]    = sum_{n,i,j} dy[n][c][i][j] * x~[n][c][i + a - r][j + b - r]
//
// Design (one CTA of 8 warps per 64 x 128 or 32 x 128 output tile):
//  * The input tile and its halo are staged once into shared memory in the
//    storage type (FP32 or BF16) with asynchronous cp.async copies; the border
//    rule is applied while staging, so the compute loops never branch on
//    coordinates.  BF16 is widened to FP32 when a row enters registers.  The
//    column halo is rounded up to 4 so every staged row stays 16-byte (FP32)
//    or 8-byte (BF16) aligned.
//  * Each lane owns 4 adjacent output columns and PY rows.  The filter is
//    consumed A rows at a time with those A rows held in registers; every
//    staged input row is read once per group with 128-bit shared loads and
//    feeds A * 4 * K FMAs (a register sliding window over rows), which keeps
//    the FMA:shared-load ratio above the 4:1 needed to stay FMA-bound.
//  * The filter gradient keeps a lane's 8 x 4 block of dy in registers and
//    streams staged x rows past it; each warp owns a fixed group of filter
//    rows whose FP32 accumulators persist across all tiles of the CTA, so the
//    cross-lane reduction (warp shuffles) runs once per CTA.  In the fused
//    backward pass, warps 0-3 compute the input gradient and warps 4-7 the
//    filter gradient of the same staged tile, so dy and x are read once.
#pragma once

#include "common.cuh"

namespace giga {

template <int K>
struct Geo {
  static constexpr int R = (K - 1) / 2;
  static constexpr int RP = (R + 3) / 4 * 4;        // column halo rounded up to 4
  static constexpr int SP = kTileW + 2 * RP;        // staged row pitch (elements)
  static constexpr int OFF = RP - R;                // first column a lane needs
  static constexpr int NV = (OFF + K + 2) / 4 + 1;  // float4 loads per lane per row
  static constexpr int KP = (K + 3) / 4 * 4;         // staged filter row pitch
  static constexpr int WPAD = K * KP;               // staged filter (floats)
};

// Filter rows held in registers per pass of the forward-style loop.
template <int K>
constexpr int fwd_group_rows() {
  return K <= 7 ? K : (K <= 15 ? 3 : (K <= 23 ? 2 : 1));
}

// Number of filter-row groups the filter-gradient warps split the taps into.
template <int K>
constexpr int dw_groups() {
  return K <= 7 ? 1 : (K <= 11 ? 2 : 4);
}

constexpr int kBwdTileH = 64;

__device__ __forceinline__ void cta_barrier() { asm volatile("bar.sync 0;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// cp.async with zero fill: src_bytes = 0 writes zeros and reads nothing.
__device__ __forceinline__ void cp_async16(float* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Wait for this thread's staging copies, then for the whole CTA.
__device__ __forceinline__ void stage_wait() {
  cp_async_wait_all();
  cta_barrier();
}

// A 16-byte shared load the compiler may not re-issue: the value must stay
// in registers (used for filter taps and dy blocks that feed many FMAs).
__device__ __forceinline__ float4 lds128_pinned(const float* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(smem_addr(p)));
  return v;
}

// Shared-memory tile element access: 4 consecutive staged elements -> FP32.
template <typename T> struct Tile;
template <> struct Tile<float> {
  static __device__ __forceinline__ float4 load4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  static __device__ __forceinline__ float4 load4_pinned(const float* p) { return lds128_pinned(p); }
  static __device__ __forceinline__ void store4(float* p, float4 v) {
    *reinterpret_cast<float4*>(p) = v;
  }
};
__device__ __forceinline__ float4 bf16x4_to_float4(uint32_t lo, uint32_t hi) {
  return make_float4(__uint_as_float(lo << 16), __uint_as_float(lo & 0xffff0000u),
                     __uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
}
template <> struct Tile<__nv_bfloat16> {
  static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    return bf16x4_to_float4(u.x, u.y);
  }
  static __device__ __forceinline__ float4 load4_pinned(const __nv_bfloat16* p) {
    uint32_t lo, hi;
    asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(smem_addr(p)));
    return bf16x4_to_float4(lo, hi);
  }
  // values come from BF16 storage, so the round trip is exact
  static __device__ __forceinline__ void store4(__nv_bfloat16* p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
  }
};

// One staged chunk of 4 consecutive columns at (gi, gj..gj+3), border applied.
template <typename T>
__device__ __forceinline__ float4 load_chunk(const T* __restrict__ plane, int H, int W, int gi,
                                             int gj, bool clamp, bool vec) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  bool row_ok = gi >= 0 && gi < H;
  if (!row_ok && clamp) {
    gi = gi < 0 ? 0 : H - 1;
    row_ok = true;
  }
  if (row_ok) {
    const T* src = plane + (int64_t)gi * W;
    if (vec && gj >= 0 && gj + 3 < W) {
      v = Elem<T>::load4(src + gj);
    } else {
      float e[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int j = gj + q;
        bool ok = j >= 0 && j < W;
        if (!ok && clamp) {
          j = j < 0 ? 0 : W - 1;
          ok = true;
        }
        e[q] = ok ? Elem<T>::load(src + j) : 0.f;
      }
      v = make_float4(e[0], e[1], e[2], e[3]);
    }
  }
  return v;
}

// Stage rows [ty0 - HR, ty0 - HR + rows) x cols [tx0 - HC, tx0 - HC + pitch)
// of one image plane into shared memory (same element type as the tensor).
// Outside the image: zero, or (clamp) the nearest edge pixel, row and column
// clamped independently.  Chunks of 4 elements that lie inside the image on
// an aligned row are asynchronous cp.async copies (16 bytes FP32, 8 bytes
// BF16); rows outside a zero border are zero-filled by cp.async; the rest
// (edges, clamped columns, unaligned rows) go element by element (FP32:
// 4-byte cp.async; BF16: a plain load and store).  Completion: stage_wait().
template <typename T, int HR, int HC, int PITCH, int NT = kThreads>
__device__ __forceinline__ void stage_tile(T* __restrict__ sm, const T* __restrict__ plane,
                                           int H, int W, int ty0, int tx0, int rows,
                                           bool clamp, bool vec) {
  constexpr int CPR = PITCH / 4;
  const int total = rows * CPR;
  for (int k = threadIdx.x; k < total; k += NT) {
    const int sr = k / CPR;
    const int sc = (k - sr * CPR) * 4;
    int gi = ty0 - HR + sr;
    const int gj = tx0 - HC + sc;
    T* dst = sm + sr * PITCH + sc;
    bool row_ok = gi >= 0 && gi < H;
    if (!row_ok && clamp) {
      gi = gi < 0 ? 0 : H - 1;
      row_ok = true;
    }
    if constexpr (sizeof(T) == 4) {
      if (!row_ok) {
        cp_async16(reinterpret_cast<float*>(dst), plane, false);
        continue;
      }
      const T* src = plane + (int64_t)gi * W;
      if (vec && gj >= 0 && gj + 3 < W) {
        cp_async16(reinterpret_cast<float*>(dst), src + gj, true);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int j = gj + q;
          bool ok = j >= 0 && j < W;
          if (!ok && clamp) {
            j = j < 0 ? 0 : W - 1;
            ok = true;
          }
          cp_async4(reinterpret_cast<float*>(dst) + q, ok ? src + j : plane, ok);
        }
      }
    } else {
      if (!row_ok) {
        cp_async8(dst, plane, false);
        continue;
      }
      const T* src = plane + (int64_t)gi * W;
      if (vec && gj >= 0 && gj + 3 < W) {
        cp_async8(dst, src + gj, true);
      } else {
        Tile<T>::store4(dst, load_chunk<T>(plane, H, W, gi, gj, clamp, vec));
      }
    }
  }
  cp_async_commit();
}

// Stage a K x K filter asynchronously (4-byte cp.async; padding columns are
// zero-filled by the same copies), optionally rotated by 180 degrees.
template <int K>
__device__ __forceinline__ void stage_filter_async(float* __restrict__ sm,
                                                   const float* __restrict__ w, bool flip,
                                                   int NT) {
  constexpr int KP = Geo<K>::KP;
  for (int k = threadIdx.x; k < K * KP; k += NT) {
    const int a = k / KP, b = k - (k / KP) * KP;
    const bool ok = b < K;
    cp_async4(sm + k, ok ? w + (flip ? (K - 1 - a) * K + (K - 1 - b) : a * K + b) : w, ok);
  }
}

// Stage a K x K filter with rows padded to KP (zeros), optionally rotated by
// 180 degrees (the input gradient's flipped filter).
template <int K>
__device__ __forceinline__ void stage_filter(float* __restrict__ sm, const float* __restrict__ w,
                                             bool flip, int NT) {
  constexpr int KP = Geo<K>::KP;
  for (int k = threadIdx.x; k < K * KP; k += NT) {
    const int a = k / KP, b = k - (k / KP) * KP;
    sm[k] = b < K ? w[flip ? (K - 1 - a) * K + (K - 1 - b) : a * K + b] : 0.f;
  }
}

// Write a lane's PY x 4 block (rows gi0.., columns gj..gj+3) with bounds checks.
template <typename T, int PY>
__device__ __forceinline__ void store_block(T* __restrict__ plane, int H, int W, int gi0, int gj,
                                            bool vec, const float (&acc)[PY][4]) {
#pragma unroll
  for (int py = 0; py < PY; ++py) {
    const int gi = gi0 + py;
    if (gi >= H) break;
    T* dst = plane + (int64_t)gi * W + gj;
    if (vec && gj + 3 < W) {
      Elem<T>::store4(dst, make_float4(acc[py][0], acc[py][1], acc[py][2], acc[py][3]));
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (gj + q < W) Elem<T>::store(dst + q, acc[py][q]);
    }
  }
}

template <int K, typename TS>
__device__ __forceinline__ void load_window_row(const TS* __restrict__ row,
                                                float (&buf)[4 * Geo<K>::NV]) {
#pragma unroll
  for (int v = 0; v < Geo<K>::NV; ++v) {
    const float4 t = Tile<TS>::load4(row + 4 * v);
    buf[4 * v + 0] = t.x;
    buf[4 * v + 1] = t.y;
    buf[4 * v + 2] = t.z;
    buf[4 * v + 3] = t.w;
  }
}

// acc[py][px] += sum_{s < A, b < K} f[s*KP + b] * win[(py + s) * SP + OFF + px + b]
// `win` points at the staged row of output row 0 plus filter row 0 of this
// group, at the lane's first column; `f` at filter row 0 of this group.
template <int K, int PY, int A, typename TS>
__device__ __forceinline__ void fwd_group(const TS* __restrict__ win,
                                          const float* __restrict__ f, float (&acc)[PY][4]) {
  using G = Geo<K>;
  float wr[A][G::KP];
#pragma unroll
  for (int s = 0; s < A; ++s)
#pragma unroll
    for (int b = 0; b < G::KP; b += 4) {
      const float4 t = lds128_pinned(f + s * G::KP + b);
      wr[s][b] = t.x;
      wr[s][b + 1] = t.y;
      wr[s][b + 2] = t.z;
      wr[s][b + 3] = t.w;
    }
#pragma unroll
  for (int ir = 0; ir < PY + A - 1; ++ir) {
    float buf[4 * G::NV];
    load_window_row<K, TS>(win + ir * G::SP, buf);
#pragma unroll
    for (int s = 0; s < A; ++s) {
      const int py = ir - s;
      if (py >= 0 && py < PY) {
#pragma unroll
        for (int b = 0; b < K; ++b)
#pragma unroll
          for (int px = 0; px < 4; ++px)
            acc[py][px] = fmaf(wr[s][b], buf[G::OFF + px + b], acc[py][px]);
      }
    }
  }
}

template <int K, int PY, typename TS>
__device__ __forceinline__ void fwd_block(const TS* __restrict__ win,
                                          const float* __restrict__ f, float (&acc)[PY][4]) {
  constexpr int A = fwd_group_rows<K>();
  constexpr int NG = K / A;
  constexpr int REM = K % A;
#pragma unroll
  for (int py = 0; py < PY; ++py)
#pragma unroll
    for (int px = 0; px < 4; ++px) acc[py][px] = 0.f;
#pragma unroll 1
  for (int g = 0; g < NG; ++g)
    fwd_group<K, PY, A, TS>(win + g * A * Geo<K>::SP, f + g * A * Geo<K>::KP, acc);
  if constexpr (REM > 0)
    fwd_group<K, PY, REM, TS>(win + NG * A * Geo<K>::SP, f + NG * A * Geo<K>::KP, acc);
}

// Filter gradient of one DR-row dy block for the filter rows [a_lo, a_lo + nrows):
// acc[s][b] += sum_{py, px} dy[py][px] * x~[py + a_lo + s][px + b]   (tile-local)
// `dyb` points at the staged dy of block row 0 (lane column), `xw` at the
// staged x row (block row 0 + a_lo) at the lane's first column.
template <int K, int AT, int DYP, int DR, typename TS>
__device__ __forceinline__ void dw_block(const TS* __restrict__ dyb,
                                         const TS* __restrict__ xw, int nrows,
                                         float (&acc)[AT][K]) {
  using G = Geo<K>;
  float d[DR][4];
#pragma unroll
  for (int py = 0; py < DR; ++py) {
    const float4 t = Tile<TS>::load4_pinned(dyb + py * DYP);
    d[py][0] = t.x;
    d[py][1] = t.y;
    d[py][2] = t.z;
    d[py][3] = t.w;
  }
#pragma unroll
  for (int ir = 0; ir < DR + AT - 1; ++ir) {
    if (ir >= DR + nrows - 1) break;
    float buf[4 * G::NV];
    load_window_row<K, TS>(xw + ir * G::SP, buf);
#pragma unroll
    for (int s = 0; s < AT; ++s) {
      const int py = ir - s;
      if (py >= 0 && py < DR && s < nrows) {
#pragma unroll
        for (int b = 0; b < K; ++b)
#pragma unroll
          for (int px = 0; px < 4; ++px)
            acc[s][b] = fmaf(d[py][px], buf[G::OFF + px + b], acc[s][b]);
      }
    }
  }
}

// Rows per unrolled block in the backward roles: the input-gradient and the
// filter-gradient warps run different unrolled bodies on the same SM, so for
// K >= 7 both use 4-row blocks to keep the two bodies within the
// instruction cache together.
template <int K>
constexpr int bwd_block_rows() {
  return K <= 5 ? 8 : 4;
}

// ---------------------------------------------------------------- forward
// Persistent: CTA b handles tiles b, b + G, b + 2G, ... (G = gridDim.x, so
// neighbouring CTAs work on neighbouring tiles at the same time and share
// halos in L2), each (kWarps * PY) x 128 pixels of one plane.  Two stages of
// shared memory: while a tile is computed, the cp.async copies of the next
// tile and of its plane's filter are in flight.  With flip = 1 the filter is
// rotated by 180 degrees: that computes g (input gradient, zero border) from dy.
template <int K, int PY, typename T>
struct FwdShape {
  using G = Geo<K>;
  static constexpr int TH = kWarps * PY;
  static constexpr int TILE_BYTES = (TH + 2 * G::R) * G::SP * (int)sizeof(T);
  static constexpr int STAGE_BYTES = G::WPAD * 4 + TILE_BYTES;  // filter, then tile
  static constexpr int SM_BYTES = 2 * STAGE_BYTES;
};

template <typename T, int K, int PY>
__global__ void __launch_bounds__(kThreads) dw_fwd_kernel(const T* __restrict__ x,
                                                          const float* __restrict__ w,
                                                          T* __restrict__ y, int C, int H, int W,
                                                          int tiles_x, int tiles_y,
                                                          int64_t num_tiles, int clamp, int vec,
                                                          int flip) {
  using G = Geo<K>;
  using S = FwdShape<K, PY, T>;
  constexpr int TH = S::TH;
  extern __shared__ __align__(16) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  auto stage = [&](int64_t t, int sb) {
    const int tx = (int)(t % tiles_x);
    const int64_t t2 = t / tiles_x;
    const int ty = (int)(t2 % tiles_y);
    const int64_t plane = t2 / tiles_y;
    float* sw = reinterpret_cast<float*>(sm + sb * S::STAGE_BYTES);
    T* sx = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES + G::WPAD * 4);
    stage_filter_async<K>(sw, w + (int64_t)(plane % C) * K * K, flip != 0, kThreads);
    stage_tile<T, G::R, G::RP, G::SP>(sx, x + plane * (int64_t)H * W, H, W, ty * TH,
                                      tx * kTileW, TH + 2 * G::R, clamp != 0, vec != 0);
  };

  int64_t t = blockIdx.x;
  if (t >= num_tiles) return;
  stage(t, 0);
  for (int sb = 0; t < num_tiles; t += gridDim.x, sb ^= 1) {
    const int64_t tn = t + gridDim.x;
    if (tn < num_tiles) {
      stage(tn, sb ^ 1);  // the other stage was released by the barrier below
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    cta_barrier();
    const int tx = (int)(t % tiles_x);
    const int64_t t2 = t / tiles_x;
    const int ty = (int)(t2 % tiles_y);
    const int64_t plane = t2 / tiles_y;
    const float* sw = reinterpret_cast<const float*>(sm + sb * S::STAGE_BYTES);
    const T* sx = reinterpret_cast<const T*>(sm + sb * S::STAGE_BYTES + G::WPAD * 4);
    float acc[PY][4];
    fwd_block<K, PY, T>(sx + warp * PY * G::SP + 4 * lane, sw, acc);
    store_block<T, PY>(y + plane * (int64_t)H * W, H, W, ty * TH + warp * PY,
                       tx * kTileW + 4 * lane, vec != 0, acc);
    cta_barrier();  // every warp is done with stage sb before it is refilled
  }
}

// -------------------------------------------------------------- backward
// MODE 0: fused; warps 0-3 write g (= dx for the zero border) from the staged
//         dy tile, warps 4-7 accumulate dw from the staged x and dy tiles.
// MODE 1: filter gradient only; all 8 warps accumulate dw (dy staged without
//         a halo).
// A CTA owns `tpc` consecutive 64 x 128 tiles of one plane and writes one
// K*K vector of FP32 partial sums to partials[blockIdx.x].
template <int K, int MODE, typename T>
struct BwdShape {
  using G = Geo<K>;
  static constexpr int NDX = MODE == 0 ? 4 : 0;
  static constexpr int NDW = kWarps - NDX;
  static constexpr int GT = dw_groups<K>();
  static constexpr int WPG = NDW / GT;              // warps per filter-row group
  static constexpr int AT = (K + GT - 1) / GT;      // max filter rows per group
  static constexpr int DW_ROWS = kBwdTileH / WPG;   // tile rows per dw warp
  static constexpr int X_ROWS = kBwdTileH + 2 * G::R;
  static constexpr int DY_HR = MODE == 0 ? G::R : 0;
  static constexpr int DY_HC = MODE == 0 ? G::RP : 0;
  static constexpr int DY_P = MODE == 0 ? G::SP : kTileW;
  static constexpr int DY_ROWS = kBwdTileH + 2 * DY_HR;
  // byte offsets: staged tiles in the storage type, filter and reduction FP32
  static constexpr int SM_X = 0;
  static constexpr int SM_DY = X_ROWS * G::SP * (int)sizeof(T);
  static constexpr int SM_W = SM_DY + DY_ROWS * DY_P * (int)sizeof(T);
  static constexpr int SM_RED = SM_W + G::WPAD * 4;
  static constexpr int SM_BYTES = SM_RED + NDW * AT * K * 4;
  static_assert(NDW % GT == 0, "filter-row groups must divide the dw warps");
  static_assert(kBwdTileH % (WPG * 8) == 0, "dw warps own whole 8-row blocks");
  static_assert(16 % bwd_block_rows<K>() == 0, "input-gradient warps own 16 rows");
};

__device__ __forceinline__ int group_lo(int g, int K, int GT) { return g * K / GT; }

// CTAs per SM the backward kernel is compiled for: the small-K instances are
// memory-bound and need fewer registers, so a third CTA adds loads in flight.
template <typename T, int K>
constexpr int bwd_min_ctas() {
  return K <= 5 ? 3 : 2;
}

template <typename T, int K, int MODE>
__global__ void __launch_bounds__(kThreads, bwd_min_ctas<T, K>())
    dw_bwd_kernel(const T* __restrict__ x, const T* __restrict__ dy, const float* __restrict__ w,
                  T* __restrict__ dx, float* __restrict__ partials, int C, int H, int W,
                  int tiles_x, int tiles_per_plane, int chunks_per_plane, int tpc, int clamp,
                  int vec) {
  using G = Geo<K>;
  using S = BwdShape<K, MODE, T>;
  extern __shared__ __align__(16) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  T* sm_x = reinterpret_cast<T*>(sm + S::SM_X);
  T* sm_dy = reinterpret_cast<T*>(sm + S::SM_DY);
  float* sm_w = reinterpret_cast<float*>(sm + S::SM_W);
  float* sm_red = reinterpret_cast<float*>(sm + S::SM_RED);

  const int64_t plane = blockIdx.x / chunks_per_plane;
  const int chunk = blockIdx.x % chunks_per_plane;
  const int t_begin = chunk * tpc;
  const int t_end = min(t_begin + tpc, tiles_per_plane);
  const int c = (int)(plane % C);
  const int64_t plane_off = plane * (int64_t)H * W;
  const T* xp = x + plane_off;
  const T* dyp = dy + plane_off;

  if (MODE == 0) stage_filter<K>(sm_w, w + (int64_t)c * K * K, true, kThreads);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp < S::NDX) {
    // ---- input-gradient warps: 16 rows each, two passes of 8 rows
    for (int t = t_begin; t < t_end; ++t) {
      const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
      cta_barrier();
      stage_tile<T, G::R, G::RP, G::SP>(sm_x, xp, H, W, ty0, tx0, S::X_ROWS, clamp != 0,
                                        vec != 0);
      stage_tile<T, S::DY_HR, S::DY_HC, S::DY_P>(sm_dy, dyp, H, W, ty0, tx0, S::DY_ROWS, false,
                                                 vec != 0);
      stage_wait();
      constexpr int BR = bwd_block_rows<K>();
#pragma unroll 1
      for (int pass = 0; pass < 16 / BR; ++pass) {
        const int r0 = warp * 16 + pass * BR;
        float acc[BR][4];
        fwd_block<K, BR, T>(sm_dy + r0 * S::DY_P + 4 * lane, sm_w, acc);
        store_block<T, BR>(dx + plane_off, H, W, ty0 + r0, tx0 + 4 * lane, vec != 0, acc);
      }
    }
    cta_barrier();
    cta_barrier();
  } else {
    // ---- filter-gradient warps
    const int wi = warp - S::NDX;
    const int g = wi % S::GT;
    const int part = wi / S::GT;
    const int a_lo = group_lo(g, K, S::GT);
    const int nrows = group_lo(g + 1, K, S::GT) - a_lo;
    float acc[S::AT][K];
#pragma unroll
    for (int s = 0; s < S::AT; ++s)
#pragma unroll
      for (int b = 0; b < K; ++b) acc[s][b] = 0.f;
    for (int t = t_begin; t < t_end; ++t) {
      const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
      cta_barrier();
      stage_tile<T, G::R, G::RP, G::SP>(sm_x, xp, H, W, ty0, tx0, S::X_ROWS, clamp != 0,
                                        vec != 0);
      stage_tile<T, S::DY_HR, S::DY_HC, S::DY_P>(sm_dy, dyp, H, W, ty0, tx0, S::DY_ROWS, false,
                                                 vec != 0);
      stage_wait();
      constexpr int BR = bwd_block_rows<K>();
#pragma unroll 1
      for (int r0 = part * S::DW_ROWS; r0 < (part + 1) * S::DW_ROWS; r0 += BR) {
        dw_block<K, S::AT, S::DY_P, BR, T>(
            sm_dy + (r0 + S::DY_HR) * S::DY_P + S::DY_HC + 4 * lane,
            sm_x + (r0 + a_lo) * G::SP + 4 * lane, nrows, acc);
      }
    }
    // warp reduction (fixed butterfly order), one row of sm_red per warp
    cta_barrier();
#pragma unroll
    for (int s = 0; s < S::AT; ++s)
#pragma unroll
      for (int b = 0; b < K; ++b) {
        float v = acc[s][b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm_red[(wi * S::AT + s) * K + b] = v;
      }
    cta_barrier();
  }
  // CTA partial for every tap, summed over the warps of its group in a fixed order.
  for (int k = threadIdx.x; k < K * K; k += kThreads) {
    const int a = k / K, b = k - (k / K) * K;
    int g = 0;
    while (g + 1 < S::GT && group_lo(g + 1, K, S::GT) <= a) ++g;
    const int s = a - group_lo(g, K, S::GT);
    float sum = 0.f;
    for (int p = 0; p < S::WPG; ++p) sum += sm_red[((p * S::GT + g) * S::AT + s) * K + b];
    partials[(int64_t)blockIdx.x * K * K + k] = sum;
  }
}

}  // namespace giga
