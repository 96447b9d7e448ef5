// dw_kernels.cuh -- depthwise K x K filtering kernels (forward, input
// gradient, filter gradient) for sm_103a.
//
// Operation (GigaAPI paper, Section 4.2.4 "Sharpening", widened to odd K,
// depthwise channels, zero/clamp borders and both gradients):
//   y[n][c][i][j]  = sum_{a,b} w[c][a][b] * x~[n][c][i + a - r][j + b - r]
//   g[n][c][u][v]  = sum_{a,b} w[c][K-1-a][K-1-b] * dy~[n][c][u + a - r][v + b - r]
//                    (dy~ zero outside the image; dx = g for the zero border,
//                    the clamp border adds the edge fold of dw_misc.cu:
//                    dw_fold_rows_kernel / dw_fold_cols_kernel in FP32,
//                    dw_fixup_kernel with dw_fold.cuh in BF16)
//   dw[c][a][b]    = sum_{n,i,j} dy[n][c][i][j] * x~[n][c][i + a - r][j + b - r]
//
// Design (one CTA of 8 warps per 64 x 128 or 32 x 128 output tile):
//  * The input tile and its halo are staged once into shared memory in the
//    storage type (FP32 or BF16).  When a plane's base and row stride are
//    16-byte aligned, one thread issues a TMA tensor load per tile (the
//    out-of-image part arrives as zeros: the zero border; under the clamp
//    border the edge tiles are then fixed in shared memory by clamp_fix);
//    other inputs are staged by every thread's cp.async copies with the border
//    rule applied while copying.  Either way the compute loops never branch on
//    coordinates.  BF16 is widened to FP32 once per staged tile (forward and
//    fused backward) or when a row enters registers.  The column halo is
//    rounded up to 16 bytes of elements so every staged row stays 16-byte
//    aligned (TMA's rule for the x coordinate).
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
#include "tma.cuh"

namespace giga {

// Column halo of a K x K filter for elements of ES bytes: r rounded up to 16
// bytes of elements (4 FP32, 8 BF16), so a staged row starts 16-byte aligned
// in memory (TMA's rule for the x coordinate) and in shared memory.
__host__ __device__ constexpr int geo_rp(int K, int ES) {
  return ES == 2 ? ((K - 1) / 2 + 7) / 8 * 8 : ((K - 1) / 2 + 3) / 4 * 4;
}

// Tile geometry of a K x K filter for elements of ES bytes.
template <int K, int ES = 4>
struct Geo {
  static constexpr int R = (K - 1) / 2;
  static constexpr int RP = geo_rp(K, ES);
  static constexpr int SP = kTileW + 2 * RP;        // staged row pitch (elements)
  static constexpr int OFF = RP - R;                // first column a lane needs
  static constexpr int OFF4 = OFF / 4 * 4;          // whole 4-element chunks skipped
  static constexpr int OFFR = OFF - OFF4;           // offset inside the first chunk
  static constexpr int NV = (OFFR + K + 2) / 4 + 1;  // 4-element loads per lane per row
  static constexpr int KP = (K + 3) / 4 * 4;         // staged filter row pitch
  static constexpr int WPAD = K * KP;               // staged filter (floats)
};

constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }

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
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
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
    asm volatile("ld.volatile.shared.v2.b32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi)
                 : "r"(smem_addr(p)));
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

// Four consecutive FP32 elements inside an image row whose start is not
// 16-byte aligned (W not a multiple of 4, or a view): the widest copies the
// source address allows -- one 16-byte copy on the rows that happen to be
// aligned, two 8-byte copies on 8-byte boundaries (every row when W = 2 mod 4,
// half of them when W is odd), else four 4-byte copies.  `dst` is 16-byte
// aligned.
__device__ __forceinline__ void stage_chunk_unaligned(float* dst, const float* src) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  if ((a & 15) == 0) {
    cp_async16(dst, src, true);
  } else if ((a & 7) == 0) {
    cp_async8(dst, src, true);
    cp_async8(dst + 2, src + 2, true);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) cp_async4(dst + q, src + q, true);
  }
}

// Stage rows [ty0 - HR, ty0 - HR + rows) x cols [tx0 - HC, tx0 - HC + pitch)
// of one image plane into shared memory (same element type as the tensor).
// Outside the image: zero, or (clamp) the nearest edge pixel, row and column
// clamped independently.  Chunks of 4 elements that lie inside the image on
// an aligned row are asynchronous cp.async copies (16 bytes FP32, 8 bytes
// BF16); rows outside a zero border are zero-filled by cp.async; the rest
// (edges, clamped columns, unaligned rows) go element by element (FP32:
// 4-byte cp.async; BF16: a plain load and store).  Completion: stage_wait().
template <typename T, int HR, int HC, int PITCH, int NT = kThreads, bool COMMIT = true>
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
      } else if (gj >= 0 && gj + 3 < W) {
        stage_chunk_unaligned(reinterpret_cast<float*>(dst), src + gj);
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
      } else if (gj >= 0 && gj + 3 < W &&
                 (reinterpret_cast<uintptr_t>(src + gj) & 3) == 0) {
        // interior chunk of a row that is not 8-byte aligned, at a 4-byte
        // boundary: two 4-byte copies of two elements each
        cp_async4(reinterpret_cast<float*>(dst), src + gj, true);
        cp_async4(reinterpret_cast<float*>(dst) + 1, src + gj + 2, true);
      } else {
        Tile<T>::store4(dst, load_chunk<T>(plane, H, W, gi, gj, clamp, vec));
      }
    }
  }
  if (COMMIT) cp_async_commit();
}

// stage_tile with the halo and pitch known only at run time (used where the
// next tile's filter size is data-dependent); issues the copies, no commit.
template <typename T, int NT>
__device__ __forceinline__ void stage_tile_rt(T* __restrict__ sm, const T* __restrict__ plane,
                                              int H, int W, int ty0, int tx0, int rows, int HR,
                                              int HC, int pitch, bool clamp, bool vec) {
  const int cpr = pitch / 4;
  const int total = rows * cpr;
  for (int k = threadIdx.x; k < total; k += NT) {
    const int sr = k / cpr;
    const int sc = (k - sr * cpr) * 4;
    int gi = ty0 - HR + sr;
    const int gj = tx0 - HC + sc;
    T* dst = sm + sr * pitch + sc;
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
      } else if (gj >= 0 && gj + 3 < W) {
        stage_chunk_unaligned(reinterpret_cast<float*>(dst), src + gj);
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
      } else if (gj >= 0 && gj + 3 < W &&
                 (reinterpret_cast<uintptr_t>(src + gj) & 3) == 0) {
        // interior chunk of a row that is not 8-byte aligned, at a 4-byte
        // boundary: two 4-byte copies of two elements each
        cp_async4(reinterpret_cast<float*>(dst), src + gj, true);
        cp_async4(reinterpret_cast<float*>(dst) + 1, src + gj + 2, true);
      } else {
        Tile<T>::store4(dst, load_chunk<T>(plane, H, W, gi, gj, clamp, vec));
      }
    }
  }
}

// A K x K filter (K known at run time) with rows padded to a multiple of 4
// (zeros), optionally rotated by 180 degrees; cp.async, no commit.
template <int NT>
__device__ __forceinline__ void stage_filter_rt(float* __restrict__ sm,
                                                const float* __restrict__ w, int K, bool flip) {
  const int kp = (K + 3) / 4 * 4;
  for (int k = threadIdx.x; k < K * kp; k += NT) {
    const int a = k / kp, b = k - (k / kp) * kp;
    const bool ok = b < K;
    cp_async4(sm + k, ok ? w + (flip ? (K - 1 - a) * K + (K - 1 - b) : a * K + b) : w, ok);
  }
}

// Staged-tile layout of storage type T in a buffer sized for the FP32 tile of
// ROWS x SPD elements: FP32 tiles are staged in place; a BF16 tile of ROWS x
// SPS elements is staged at the end of the buffer (128-byte aligned for TMA)
// and widened into the FP32 layout at the start by widen_tile, so every
// compute path reads FP32 tiles.
template <typename T, int ROWS, int SPD, int SPS>
struct StagedTile {
  static constexpr int BYTES = round_up(ROWS * SPD * 4, 128);  // the FP32 tile
  static constexpr int STAGE_BYTES = ROWS * SPS * (int)sizeof(T);
  static constexpr int STAGE_OFF = sizeof(T) == 4 ? 0 : (BYTES - STAGE_BYTES) / 128 * 128;
  static_assert(sizeof(T) == 2 || SPS == SPD, "FP32 tiles are staged in their own layout");
  static_assert(STAGE_OFF >= 0 && STAGE_OFF + STAGE_BYTES <= BYTES, "staged tile fits");
};

// Widen the BF16 tile staged at `src` (ROWS x SPS) into the FP32 tile at `dst`
// (ROWS x SPD; FP32 column c is staged column c + D).  src lies at the end of
// dst's buffer.  Chunks of 4 elements go in increasing order, PB per thread
// per pass: a pass reads its chunks into registers, the CTA synchronises, then
// it writes.  The FP32 writes of a pass never reach the staged bytes of a
// later pass (the FP32 image of chunk k ends below the staged image of every
// chunk after the pass, checked on the host for every shape in use), so only
// the barrier between a pass's reads and writes is needed; a final barrier
// publishes the FP32 tile.
template <int ROWS, int SPD, int SPS, int D, int NT>
__device__ __forceinline__ void widen_tile(float* __restrict__ dst,
                                           const __nv_bfloat16* __restrict__ src) {
  constexpr int CPR = SPD / 4;
  constexpr int TOTAL = ROWS * CPR;
  constexpr int PB = 4;
  constexpr int PASSES = (TOTAL + NT * PB - 1) / (NT * PB);
  static_assert(D % 4 == 0 && SPD % 4 == 0 && D + SPD <= SPS, "chunks stay aligned");
#pragma unroll 1
  for (int p = 0; p < PASSES; ++p) {
    uint2 v[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int k = (p * PB + i) * NT + threadIdx.x;
      if (k < TOTAL) {
        const int r = k / CPR, c = (k - (k / CPR) * CPR) * 4;
        v[i] = *reinterpret_cast<const uint2*>(src + r * SPS + c + D);
      }
    }
    cta_barrier();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int k = (p * PB + i) * NT + threadIdx.x;
      if (k < TOTAL) {
        const int r = k / CPR, c = (k - (k / CPR) * CPR) * 4;
        *reinterpret_cast<float4*>(dst + r * SPD + c) = bf16x4_to_float4(v[i].x, v[i].y);
      }
    }
  }
  cta_barrier();
}

// The halo tile of filter size K (ROWS rows) staged as T, widened if BF16.
template <int K, typename T, int ROWS>
using HaloTile = StagedTile<T, ROWS, Geo<K, 4>::SP, Geo<K, sizeof(T)>::SP>;

template <int K, int ROWS, int NT>
__device__ __forceinline__ void widen_halo_tile(float* dst, const __nv_bfloat16* src) {
  widen_tile<ROWS, Geo<K, 4>::SP, Geo<K, 2>::SP, Geo<K, 2>::RP - Geo<K, 4>::RP, NT>(dst, src);
}

// Clamp border on a tile that TMA staged with zeros outside the image: tile
// row sr is image row ty0 - HR + sr, tile column sc image column tx0 - HC + sc.
// Pass 1 gives the out-of-image columns of every in-image row the value of
// the nearest in-image column; pass 2 copies whole rows (corners included)
// from the nearest in-image row.  Every thread of the CTA calls it; it ends
// with a barrier.
template <typename T, int PITCH, int NT>
__device__ __forceinline__ void clamp_fix(T* __restrict__ sm, int H, int W, int ty0, int tx0,
                                          int HR, int HC, int rows) {
  const int c_lo = max(0, HC - tx0), c_hi = min(PITCH, W - tx0 + HC);
  const int r_lo = max(0, HR - ty0), r_hi = min(rows, H - ty0 + HR);
  const int nl = c_lo, nr = PITCH - c_hi, ncol = nl + nr;
  if (ncol > 0) {
    const int total = (r_hi - r_lo) * ncol;
    for (int k = threadIdx.x; k < total; k += NT) {
      const int r = r_lo + k / ncol, c = k - (k / ncol) * ncol;
      T* row = sm + r * PITCH;
      if (c < nl)
        row[c] = row[c_lo];
      else
        row[c_hi + (c - nl)] = row[c_hi - 1];
    }
    cta_barrier();
  }
  const int nt = r_lo, nb = rows - r_hi;
  if (nt + nb > 0) {
    const int total = (nt + nb) * PITCH;
    for (int k = threadIdx.x; k < total; k += NT) {
      const int r = k / PITCH, c = k - (k / PITCH) * PITCH;
      const int dst = r < nt ? r : r_hi + (r - nt);
      const int src = r < nt ? r_lo : r_hi - 1;
      sm[dst * PITCH + c] = sm[src * PITCH + c];
    }
  }
  cta_barrier();
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

// The window of a lane's 4 output columns: staged columns from the lane's
// first column + OFF4 on (buf[OFFR + px + b] is input column px + b - r).
template <int K, typename TS>
__device__ __forceinline__ void load_window_row(const TS* __restrict__ row,
                                                float (&buf)[4 * Geo<K, sizeof(TS)>::NV]) {
  using G = Geo<K, sizeof(TS)>;
#pragma unroll
  for (int v = 0; v < G::NV; ++v) {
    const float4 t = Tile<TS>::load4(row + G::OFF4 + 4 * v);
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
  using G = Geo<K, sizeof(TS)>;
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
            acc[py][px] = fmaf(wr[s][b], buf[G::OFFR + px + b], acc[py][px]);
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
    fwd_group<K, PY, A, TS>(win + g * A * Geo<K, sizeof(TS)>::SP, f + g * A * Geo<K>::KP, acc);
  if constexpr (REM > 0)
    fwd_group<K, PY, REM, TS>(win + NG * A * Geo<K, sizeof(TS)>::SP, f + NG * A * Geo<K>::KP, acc);
}

// Filter gradient of one DR-row dy block for the NR filter rows [a_lo, a_lo + NR):
// acc[s][b] += sum_{py, px} dy[py][px] * x~[py + a_lo + s][px + b]   (tile-local)
// `dyb` points at the staged dy of block row 0 (lane column), `xw` at the
// staged x row (block row 0 + a_lo) at the lane's first column.  NR is a
// compile-time constant: the unrolled body has no data-dependent control flow
// (with a run-time row count the accumulators live across guarded paths and
// are copied where those paths merge).
template <int K, int NR, int AT, int DYP, int DR, typename TS>
__device__ __forceinline__ void dw_block(const TS* __restrict__ dyb,
                                         const TS* __restrict__ xw, float (&acc)[AT][K]) {
  static_assert(NR >= 1 && NR <= AT, "row count");
  using G = Geo<K, sizeof(TS)>;
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
  for (int ir = 0; ir < DR + NR - 1; ++ir) {
    float buf[4 * G::NV];
    load_window_row<K, TS>(xw + ir * G::SP, buf);
#pragma unroll
    for (int s = 0; s < NR; ++s) {
      const int py = ir - s;
      if (py >= 0 && py < DR) {
#pragma unroll
        for (int b = 0; b < K; ++b)
#pragma unroll
          for (int px = 0; px < 4; ++px)
            acc[s][b] = fmaf(d[py][px], buf[G::OFFR + px + b], acc[s][b]);
      }
    }
  }
}

// `nblocks` consecutive DR-row blocks for this warp's filter-row group of
// `nrows` rows.  Splitting K rows into GT groups gives groups of AT or
// AT - 1 rows; the branch on the (warp-uniform, fixed) row count is taken
// once, outside the unrolled bodies.
template <int K, int AT, int GT, int DYP, int DR, typename TS>
__device__ __forceinline__ void dw_rows(const TS* __restrict__ dyb, const TS* __restrict__ xw,
                                        int nblocks, int nrows, float (&acc)[AT][K]) {
  constexpr int SP = Geo<K, sizeof(TS)>::SP;
  if constexpr (K % GT == 0) {
#pragma unroll 1
    for (int i = 0; i < nblocks; ++i)
      dw_block<K, AT, AT, DYP, DR, TS>(dyb + i * DR * DYP, xw + i * DR * SP, acc);
  } else {
    if (nrows == AT) {
#pragma unroll 1
      for (int i = 0; i < nblocks; ++i)
        dw_block<K, AT, AT, DYP, DR, TS>(dyb + i * DR * DYP, xw + i * DR * SP, acc);
    } else {
#pragma unroll 1
      for (int i = 0; i < nblocks; ++i)
        dw_block<K, AT - 1, AT, DYP, DR, TS>(dyb + i * DR * DYP, xw + i * DR * SP, acc);
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
  using G = Geo<K>;  // FP32 compute geometry
  static constexpr int TH = kWarps * PY;
  static constexpr int ROWS = TH + 2 * G::R;
  using ST = HaloTile<K, T, ROWS>;
  static constexpr int W_OFF = ST::BYTES;  // FP32 tile (128-aligned), then the filter
  static constexpr int STAGE_BYTES = round_up(W_OFF + G::WPAD * 4, 128);
  static constexpr int HEAD = 128;  // two mbarriers and the abort flag
  static constexpr int SM_BYTES = HEAD + 2 * STAGE_BYTES;
  static constexpr int SM_BYTES_1 = HEAD + STAGE_BYTES;  // one tile per CTA
};

template <typename T, int K, int PY>
__device__ __forceinline__ void dw_fwd_body(
    const CUtensorMap& tmx, const T* __restrict__ x, const float* __restrict__ w,
    T* __restrict__ y, FastDiv fc, int H, int W, FastDiv ftx, FastDiv fty, int64_t num_tiles,
    int clamp, int vec, int flip, int use_tma, int64_t pf, int* err) {
  using G = Geo<K>;
  using GS = Geo<K, sizeof(T)>;
  using S = FwdShape<K, PY, T>;
  using ST = typename S::ST;
  constexpr int TH = S::TH;
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // tile t (< 2^31) -> column and row of the tile, plane (n * C + c)
  auto coords = [&](int64_t t, int& ty0, int& tx0, int& plane) {
    const uint32_t u = (uint32_t)t;
    const uint32_t r = fdiv(u, ftx);
    tx0 = (int)(u - r * ftx.d) * kTileW;
    const uint32_t pl = fdiv(r, fty);
    ty0 = (int)(r - pl * fty.d) * TH;
    plane = (int)pl;
  };
  auto stage = [&](int64_t t, int sb) {
    int ty0, tx0, plane;
    coords(t, ty0, tx0, plane);
    char* buf = sm + S::HEAD + sb * S::STAGE_BYTES;
    T* staged = reinterpret_cast<T*>(buf + ST::STAGE_OFF);
    float* sw = reinterpret_cast<float*>(buf + S::W_OFF);
    const int c = plane - (int)(fdiv((uint32_t)plane, fc) * fc.d);
    stage_filter_async<K>(sw, w + (int64_t)c * K * K, flip != 0, kThreads);
    if (use_tma) {
      cp_async_commit();
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bars + sb, (uint32_t)ST::STAGE_BYTES);
        tma_load_3d(staged, &tmx, tx0 - GS::RP, ty0 - G::R, plane, bars + sb);
      }
    } else {
      stage_tile<T, G::R, GS::RP, GS::SP>(staged, x + (int64_t)plane * H * W, H, W, ty0, tx0,
                                          S::ROWS, clamp != 0, vec != 0);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  cta_barrier();
  int64_t t = blockIdx.x;
  if (t >= num_tiles) return;
  stage(t, 0);
  uint32_t phase = 0;  // bit s: parity of the next TMA completion on stage s
  int sb = 0;
  for (; t < num_tiles; t += gridDim.x, sb ^= 1) {
    // L2 prefetch of the tile this CTA's successor (one tile per CTA) or this
    // CTA two tiles on (persistent) will load: its TMA load then hits L2
    if (use_tma && pf > 0 && threadIdx.x == 0 && t + pf < num_tiles) {
      int py0, px0, pplane;
      coords(t + pf, py0, px0, pplane);
      tma_prefetch_3d(&tmx, px0 - GS::RP, py0 - G::R, pplane);
    }
    const int64_t tn = t + gridDim.x;
    if (tn < num_tiles) {
      stage(tn, sb ^ 1);  // the other stage was released by the barrier below
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    if (use_tma) {
      if (!mbar_wait(bars + sb, (phase >> sb) & 1u)) {
        record_error(err, kDevErrTimeout);
        *s_abort = 1;
      }
      phase ^= 1u << sb;
    }
    cta_barrier();
    if (*s_abort) break;
    int ty0, tx0, plane;
    coords(t, ty0, tx0, plane);
    char* buf = sm + S::HEAD + sb * S::STAGE_BYTES;
    float* sx = reinterpret_cast<float*>(buf);
    const float* sw = reinterpret_cast<const float*>(buf + S::W_OFF);
    if constexpr (sizeof(T) == 2)
      widen_halo_tile<K, S::ROWS, kThreads>(
          sx, reinterpret_cast<const __nv_bfloat16*>(buf + ST::STAGE_OFF));
    if (use_tma && clamp &&
        (ty0 - G::R < 0 || ty0 + TH + G::R > H || tx0 - G::RP < 0 || tx0 + kTileW + G::RP > W))
      clamp_fix<float, G::SP, kThreads>(sx, H, W, ty0, tx0, G::R, G::RP, S::ROWS);
    float acc[PY][4];
    fwd_block<K, PY, float>(sx + warp * PY * G::SP + 4 * lane, sw, acc);
    store_block<T, PY>(y + (int64_t)plane * H * W, H, W, ty0 + warp * PY, tx0 + 4 * lane,
                       vec != 0, acc);
    cta_barrier();  // every warp is done with stage sb before it is refilled
  }
  cp_async_wait_group<0>();
  // after an abort: let a TMA load still in flight land (bounded) before exiting
  if (*s_abort && use_tma && t + gridDim.x < num_tiles)
    mbar_wait(bars + (sb ^ 1), (phase >> (sb ^ 1)) & 1u);
}

template <typename T, int K, int PY>
__global__ void __launch_bounds__(kThreads) dw_fwd_kernel(
    const __grid_constant__ CUtensorMap tmx, const T* __restrict__ x, const float* __restrict__ w,
    T* __restrict__ y, FastDiv fc, int H, int W, FastDiv ftx, FastDiv fty, int64_t num_tiles,
    int clamp, int vec, int flip, int use_tma, int64_t pf, int* err) {
  dw_fwd_body<T, K, PY>(tmx, x, w, y, fc, H, W, ftx, fty, num_tiles, clamp, vec, flip, use_tma,
                        pf, err);
}

// The same pass compiled for five CTAs per SM (at most 51 registers).  Used
// for FP32 K = 7 one tile per CTA, where it fits in 48 registers and 38.5 KB
// of shared memory and the extra CTA per SM hides more of each CTA's tile
// load; other sizes keep the default allocation (with this bound K = 3 and 15
// lose registers they need).
template <typename T, int K, int PY>
__global__ void __launch_bounds__(kThreads, 5) dw_fwd_kernel_hi_occ(
    const __grid_constant__ CUtensorMap tmx, const T* __restrict__ x, const float* __restrict__ w,
    T* __restrict__ y, FastDiv fc, int H, int W, FastDiv ftx, FastDiv fty, int64_t num_tiles,
    int clamp, int vec, int flip, int use_tma, int64_t pf, int* err) {
  dw_fwd_body<T, K, PY>(tmx, x, w, y, fc, H, W, ftx, fty, num_tiles, clamp, vec, flip, use_tma,
                        pf, err);
}

// ------------------------------------------------------ separable filter
// y[c][i][j] = sum_a wcol[c][a] * t[i + a - r][j],
// t[i][j]    = sum_b wrow[c][b] * x~[i][j + b - r]   (x~: the border applied),
// the K x K filter wcol (x) wrow applied as a row pass then a column pass:
// 2K instead of K^2 multiply-adds per pixel.  One 64 x 128 tile per CTA; the
// halo tile is staged like the forward's (TMA or cp.async, clamp fix, BF16
// widened); the row pass writes t over the first 128 columns of the same
// staged row (a warp owns whole rows and reads a row completely before it
// writes it), then the column pass runs down t in 8-row register blocks.
template <int K, typename T>
struct SepShape {
  using G = Geo<K>;
  static constexpr int TH = 64;
  static constexpr int ROWS = TH + 2 * G::R;
  using ST = HaloTile<K, T, ROWS>;
  static constexpr int HEAD = 128;  // mbarrier, abort flag
  static constexpr int W_OFF = HEAD + ST::BYTES;  // wrow then wcol, K floats each (padded)
  static constexpr int SM_BYTES = W_OFF + 2 * round_up(K, 4) * 4;
};

template <typename T, int K>
__device__ __forceinline__ void dw_sep_body(
    const CUtensorMap& tmx, const T* __restrict__ x, const float* __restrict__ wcol,
    const float* __restrict__ wrow, T* __restrict__ y, FastDiv fc, int H, int W, FastDiv ftx,
    FastDiv fty, int clamp, int vec, int use_tma, int pf, int* err) {
  using G = Geo<K>;
  using GS = Geo<K, sizeof(T)>;
  using S = SepShape<K, T>;
  using ST = typename S::ST;
  constexpr int KP = round_up(K, 4);
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  float* st = reinterpret_cast<float*>(sm + S::HEAD);
  float* swr = reinterpret_cast<float*>(sm + S::W_OFF);
  float* swc = swr + KP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x;
  const uint32_t t2 = fdiv(t, ftx);
  const int tx0 = (int)(t - t2 * ftx.d) * kTileW;
  const uint32_t pl = fdiv(t2, fty);
  const int ty0 = (int)(t2 - pl * fty.d) * S::TH;
  const int plane = (int)pl;
  const int c = (int)(pl - fdiv(pl, fc) * fc.d);

  for (int k = threadIdx.x; k < 2 * KP; k += kThreads) {
    const int b = k < KP ? k : k - KP;
    const float* src = (k < KP ? wrow : wcol) + (int64_t)c * K;
    cp_async4(swr + k, b < K ? src + b : src, b < K);
  }
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + 8);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  cta_barrier();
  T* staged = reinterpret_cast<T*>(sm + S::HEAD + ST::STAGE_OFF);
  if (use_tma) {
    cp_async_commit();
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, (uint32_t)ST::STAGE_BYTES);
      tma_load_3d(staged, &tmx, tx0 - GS::RP, ty0 - G::R, plane, bar);
      // L2 prefetch of the tile the CTA starting one wave of resident CTAs
      // later will load
      if (pf > 0 && t + (uint32_t)pf < gridDim.x) {
        const uint32_t u = t + (uint32_t)pf, u2 = fdiv(u, ftx), upl = fdiv(u2, fty);
        tma_prefetch_3d(&tmx, (int)(u - u2 * ftx.d) * kTileW - GS::RP,
                        (int)(u2 - upl * fty.d) * S::TH - G::R, (int)upl);
      }
    }
    cp_async_wait_all();
    if (!mbar_wait(bar, 0)) {
      record_error(err, kDevErrTimeout);
      *s_abort = 1;
    }
  } else {
    stage_tile<T, G::R, GS::RP, GS::SP>(staged, x + (int64_t)plane * H * W, H, W, ty0, tx0,
                                        S::ROWS, clamp != 0, vec != 0);
    cp_async_wait_all();
  }
  cta_barrier();
  if (*s_abort) {
    mbar_wait(bar, 0);  // let a late copy land (bounded) before the CTA exits
    return;
  }
  if constexpr (sizeof(T) == 2)
    widen_halo_tile<K, S::ROWS, kThreads>(st, reinterpret_cast<const __nv_bfloat16*>(staged));
  if (use_tma && clamp &&
      (ty0 - G::R < 0 || ty0 + S::TH + G::R > H || tx0 - G::RP < 0 || tx0 + kTileW + G::RP > W))
    clamp_fix<float, G::SP, kThreads>(st, H, W, ty0, tx0, G::R, G::RP, S::ROWS);

  // row pass, in place: row sr of t = columns [0, 128) of staged row sr
  for (int sr = warp; sr < S::ROWS; sr += kWarps) {
    float buf[4 * G::NV];
    load_window_row<K, float>(st + sr * G::SP + 4 * lane, buf);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const float wb = swr[b];
#pragma unroll
      for (int px = 0; px < 4; ++px) o[px] = fmaf(wb, buf[G::OFFR + px + b], o[px]);
    }
    __syncwarp();  // every lane has read the row before any lane overwrites it
    *reinterpret_cast<float4*>(st + sr * G::SP + 4 * lane) = make_float4(o[0], o[1], o[2], o[3]);
  }
  cta_barrier();

  // column pass: warp w owns output rows 8w .. 8w + 7
  constexpr int PY = 8;
  float acc[PY][4];
#pragma unroll
  for (int py = 0; py < PY; ++py)
#pragma unroll
    for (int px = 0; px < 4; ++px) acc[py][px] = 0.f;
#pragma unroll
  for (int ir = 0; ir < PY + K - 1; ++ir) {
    const float4 v = *reinterpret_cast<const float4*>(st + (warp * PY + ir) * G::SP + 4 * lane);
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const int py = ir - a;
      if (py >= 0 && py < PY) {
        const float wa = swc[a];
        acc[py][0] = fmaf(wa, v.x, acc[py][0]);
        acc[py][1] = fmaf(wa, v.y, acc[py][1]);
        acc[py][2] = fmaf(wa, v.z, acc[py][2]);
        acc[py][3] = fmaf(wa, v.w, acc[py][3]);
      }
    }
  }
  store_block<T, PY>(y + (int64_t)plane * H * W, H, W, ty0 + warp * PY, tx0 + 4 * lane,
                     vec != 0, acc);
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) dw_sep_kernel(
    const __grid_constant__ CUtensorMap tmx, const T* __restrict__ x,
    const float* __restrict__ wcol, const float* __restrict__ wrow, T* __restrict__ y, FastDiv fc,
    int H, int W, FastDiv ftx, FastDiv fty, int clamp, int vec, int use_tma, int pf, int* err) {
  dw_sep_body<T, K>(tmx, x, wcol, wrow, y, fc, H, W, ftx, fty, clamp, vec, use_tma, pf, err);
}

// The same pass compiled for five CTAs per SM (48 registers): used for FP32
// K = 13 and 15, whose tiles (44 KB) still fit five times in shared memory and
// whose pass waits on its tile loads (K = 15: 0.701 -> 0.689 ms on
// 8 x 3 x 4096^2); smaller K run near the HBM rate with the default allocation.
template <typename T, int K>
__global__ void __launch_bounds__(kThreads, 5) dw_sep_kernel_hi_occ(
    const __grid_constant__ CUtensorMap tmx, const T* __restrict__ x,
    const float* __restrict__ wcol, const float* __restrict__ wrow, T* __restrict__ y, FastDiv fc,
    int H, int W, FastDiv ftx, FastDiv fty, int clamp, int vec, int use_tma, int pf, int* err) {
  dw_sep_body<T, K>(tmx, x, wcol, wrow, y, fc, H, W, ftx, fty, clamp, vec, use_tma, pf, err);
}

// -------------------------------------------------------------- backward
// Fused backward: warps 0-3 write g (= dx for the zero border) from the staged
// dy tile, warps 4-7 accumulate dw from the staged x and dy tiles.  A CTA owns
// `tpc` consecutive 64 x 128 tiles of one plane and writes one K*K vector of
// FP32 partial sums to partials[blockIdx.x].  FP32 planes with a 16-byte row
// stride are staged by two TMA loads per tile (zeros outside the image; under
// the clamp border the x tile of an edge tile then gets clamp_fix), others by
// cp.async with the border applied.
template <int K, typename T>
struct BwdShape {
  using G = Geo<K>;  // FP32 compute geometry
  static constexpr int NDX = 4;
  static constexpr int NDW = kWarps - NDX;
  static constexpr int GT = dw_groups<K>();
  static constexpr int WPG = NDW / GT;              // warps per filter-row group
  static constexpr int AT = (K + GT - 1) / GT;      // max filter rows per group
  static constexpr int DW_ROWS = kBwdTileH / WPG;   // tile rows per dw warp
  static constexpr int ROWS = kBwdTileH + 2 * G::R;  // x and dy tiles, both with the halo
  using ST = HaloTile<K, T, ROWS>;
  // byte offsets: mbarrier and abort flag, the FP32 x and dy tiles (staged
  // tiles at ST::STAGE_OFF inside them, 128-byte aligned for TMA), flipped
  // filter and reduction
  static constexpr int SM_X = 128;
  static constexpr int SM_DY = SM_X + ST::BYTES;
  static constexpr int SM_W = SM_DY + ST::BYTES;
  // the warps' filter-gradient sums are written after every warp has left the
  // tile loop, so they reuse the x tile's space (3 CTAs per SM fit at K = 7)
  static constexpr int SM_RED = SM_X;
  static constexpr int SM_BYTES = SM_W + G::WPAD * 4;
  static_assert(NDW * AT * K * 4 <= ST::BYTES, "reduction rows fit the x tile");
  static_assert(NDW % GT == 0, "filter-row groups must divide the dw warps");
  static_assert(kBwdTileH % (WPG * 8) == 0, "dw warps own whole 8-row blocks");
  static_assert(16 % bwd_block_rows<K>() == 0, "input-gradient warps own 16 rows");
};

__device__ __forceinline__ int group_lo(int g, int K, int GT) { return g * K / GT; }

// CTAs per SM the backward kernel is compiled for: the small-K instances are
// memory-bound and need fewer registers, so a third CTA adds loads in flight.
template <typename T, int K>
constexpr int bwd_min_ctas() {
  return (K <= 5 || (K == 7 && sizeof(T) == 4)) ? 3 : 2;
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads, bwd_min_ctas<T, K>())
    dw_bwd_kernel(const __grid_constant__ CUtensorMap tmx,
                  const __grid_constant__ CUtensorMap tmdy, const T* __restrict__ x,
                  const T* __restrict__ dy, const float* __restrict__ w, T* __restrict__ dx,
                  float* __restrict__ partials, int C, int H, int W, int tiles_x,
                  int tiles_per_plane, int chunks_per_plane, int tpc, int clamp, int vec,
                  int use_tma, int* err) {
  using G = Geo<K>;
  using GS = Geo<K, sizeof(T)>;
  using S = BwdShape<K, T>;
  using ST = typename S::ST;
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + 8);
  float* sm_x = reinterpret_cast<float*>(sm + S::SM_X);
  float* sm_dy = reinterpret_cast<float*>(sm + S::SM_DY);
  T* st_x = reinterpret_cast<T*>(sm + S::SM_X + ST::STAGE_OFF);
  T* st_dy = reinterpret_cast<T*>(sm + S::SM_DY + ST::STAGE_OFF);
  float* sm_w = reinterpret_cast<float*>(sm + S::SM_W);
  float* sm_red = reinterpret_cast<float*>(sm + S::SM_RED);

  const int plane = (int)(blockIdx.x / (uint32_t)chunks_per_plane);
  const int chunk = (int)(blockIdx.x - (uint32_t)plane * chunks_per_plane);
  const int t_begin = chunk * tpc;
  const int t_end = min(t_begin + tpc, tiles_per_plane);
  const int c = plane % C;
  const int64_t plane_off = (int64_t)plane * H * W;
  const T* xp = x + plane_off;
  const T* dyp = dy + plane_off;

  // rotated filter; its copies complete with the first tile's
  stage_filter_async<K>(sm_w, w + (int64_t)c * K * K, true, kThreads);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  uint32_t phase = 0;
  // Stage tile (ty0, tx0) after every warp is done with the previous one;
  // false if a TMA wait gave up (every thread then leaves its tile loop).
  auto stage = [&](int ty0, int tx0) -> bool {
    cta_barrier();
    if (use_tma) {
      cp_async_commit();
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)(2 * ST::STAGE_BYTES));
        tma_load_3d(st_x, &tmx, tx0 - GS::RP, ty0 - G::R, (int)plane, bar);
        tma_load_3d(st_dy, &tmdy, tx0 - GS::RP, ty0 - G::R, (int)plane, bar);
      }
      cp_async_wait_all();
      if (mbar_wait(bar, phase))
        phase ^= 1u;
      else {
        record_error(err, kDevErrTimeout);
        *s_abort = 1;
      }
      cta_barrier();
      if (*s_abort) return false;
    } else {
      stage_tile<T, G::R, GS::RP, GS::SP>(st_x, xp, H, W, ty0, tx0, S::ROWS, clamp != 0,
                                          vec != 0);
      stage_tile<T, G::R, GS::RP, GS::SP>(st_dy, dyp, H, W, ty0, tx0, S::ROWS, false,
                                          vec != 0);
      stage_wait();
    }
    if constexpr (sizeof(T) == 2) {
      widen_halo_tile<K, S::ROWS, kThreads>(sm_x, reinterpret_cast<const __nv_bfloat16*>(st_x));
      widen_halo_tile<K, S::ROWS, kThreads>(sm_dy, reinterpret_cast<const __nv_bfloat16*>(st_dy));
    }
    if (use_tma && clamp &&
        (ty0 - G::R < 0 || ty0 + kBwdTileH + G::R > H || tx0 - G::RP < 0 ||
         tx0 + kTileW + G::RP > W))
      clamp_fix<float, G::SP, kThreads>(sm_x, H, W, ty0, tx0, G::R, G::RP, S::ROWS);
    return true;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp < S::NDX) {
    // ---- input-gradient warps: 16 rows each, in blocks of BR rows
    for (int t = t_begin; t < t_end; ++t) {
      const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
      if (!stage(ty0, tx0)) break;
      constexpr int BR = bwd_block_rows<K>();
#pragma unroll 1
      for (int pass = 0; pass < 16 / BR; ++pass) {
        const int r0 = warp * 16 + pass * BR;
        float acc[BR][4];
        fwd_block<K, BR, float>(sm_dy + r0 * G::SP + 4 * lane, sm_w, acc);
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
      if (!stage(ty0, tx0)) break;
      constexpr int BR = bwd_block_rows<K>();
      const int r0 = part * S::DW_ROWS;
      dw_rows<K, S::AT, S::GT, G::SP, BR, float>(sm_dy + (r0 + G::R) * G::SP + G::RP + 4 * lane,
                                             sm_x + (r0 + a_lo) * G::SP + 4 * lane,
                                             S::DW_ROWS / BR, nrows, acc);
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
  cp_async_wait_all();
  if (*s_abort && use_tma) mbar_wait(bar, phase);  // let a late TMA load land (bounded)
}

// ------------------------------------------------------- filter gradient
// The filter gradient alone (Eq. 3's adjoint with respect to the filter):
// dw[c][a][b] = sum over n, i, j of dy[n][c][i][j] * xs[n][c][i + a - r][j + b - r],
// xs the border-extended input.  One CTA of 12 or 16 warps per SM, persistent over
// chunks of `tpc` consecutive 64 x 128 tiles of one plane (chunk q runs on
// CTA q mod gridDim.x).  NS shared-memory stages hold {x tile with halo, dy
// tile}; the copies of the tile NS - 1 items ahead are in flight while the
// current one is reduced, across chunk boundaries too.  For FP32 rows with a
// 16-byte stride a stage is filled by two TMA tensor loads issued by one
// thread (out-of-image reads arrive as zeros: the zero border; under the
// clamp border the edge tiles then get clamp_fix); otherwise by every
// thread's cp.async copies with the border applied.  Tap rows are split into GT groups; warp w takes group w / WPG and
// tile rows part w mod WPG, so each of the SM's four schedulers (w mod 4)
// holds one warp of every group.  At the end of a chunk the warps' sums
// (fixed butterfly order) and then the group's warps (fixed order) give the
// chunk's partial for every tap.
constexpr int kFilterTileH = 64;
static_assert(kFilterTileH == kBwdTileH, "both filter-gradient kernels share the chunk layout");

// Warps and tap-row groups: K = 9 and 15 split into 3 equal groups (12 warps,
// up to 170 registers for the larger accumulator set: measured faster than 5
// groups of 3 rows on 20 warps at 96 registers); the rest use 16 warps and
// dw_groups<K>().
template <int K>
constexpr int filter_warps() {
  return (K == 9 || K == 15) ? 12 : 16;
}
template <int K>
constexpr int filter_groups() {
  return (K == 9 || K == 15) ? 3 : dw_groups<K>();
}

template <int K, typename T>
struct FilterShape {
  using G = Geo<K, sizeof(T)>;  // tiles stay in the storage type (no widening pass)
  static constexpr int NW = filter_warps<K>();
  static constexpr int NT = NW * 32;
  static constexpr int GT = filter_groups<K>();
  static constexpr int WPG = NW / GT;
  static constexpr int AT = (K + GT - 1) / GT;
  static constexpr int ROWS = kFilterTileH / WPG;  // tile rows per warp
  static constexpr int DR = 4;                     // dy rows per unrolled block
  static constexpr int X_ROWS = kFilterTileH + 2 * G::R;
  static constexpr int X_BYTES = X_ROWS * G::SP * (int)sizeof(T);
  static constexpr int DY_BYTES = kFilterTileH * kTileW * (int)sizeof(T);
  static constexpr int DY_OFF = round_up(X_BYTES, 128);  // TMA destinations: 128-byte aligned
  static constexpr int STAGE_BYTES = round_up(DY_OFF + DY_BYTES, 128);
  static constexpr int NS = K <= 9 ? 3 : 2;
  static constexpr int SM_RED = NS * STAGE_BYTES;
  static constexpr int SM_BAR = round_up(SM_RED + NW * AT * K * 4, 8);
  static constexpr int SM_BYTES = SM_BAR + NS * 8 + 8;  // mbarriers, abort flag
  static_assert(NW % GT == 0 && NW % 4 == 0 && ROWS % DR == 0, "warps own whole row blocks");
  static_assert(SM_BYTES <= 227 * 1024, "shared memory");
};

template <typename T, int K>
__global__ void __launch_bounds__(FilterShape<K, T>::NT, 1)
    dw_filter_kernel(const __grid_constant__ CUtensorMap tmx,
                     const __grid_constant__ CUtensorMap tmdy, const T* __restrict__ x,
                     const T* __restrict__ dy, float* __restrict__ partials, int H, int W,
                     FastDiv ftx, int tiles_per_plane, FastDiv fcpp, int tpc, int num_chunks,
                     int clamp, int vec, int use_tma, int* err) {
  using G = Geo<K, sizeof(T)>;
  using S = FilterShape<K, T>;
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  float* sm_red = reinterpret_cast<float*>(sm + S::SM_RED);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::SM_BAR);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + S::SM_BAR + S::NS * 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / S::WPG, part = warp % S::WPG;
  const int a_lo = group_lo(g, K, S::GT);
  const int nrows = group_lo(g + 1, K, S::GT) - a_lo;

  // (chunk, tile) items in execution order; t < t_end while valid
  // chunk q < 2^31 of plane q / chunks_per_plane; tile t of that plane is
  // tile row t / tiles_x, column t % tiles_x
  struct Item {
    int q;
    int t, t_end;
  };
  auto tile_origin = [&](int t, int& ty0, int& tx0) {
    const uint32_t r = fdiv((uint32_t)t, ftx);
    ty0 = (int)r * kFilterTileH;
    tx0 = (t - (int)(r * ftx.d)) * kTileW;
  };
  auto first_tile = [&](Item& it) {
    const int ch = it.q - (int)(fdiv((uint32_t)it.q, fcpp) * fcpp.d);
    it.t = ch * tpc;
    it.t_end = min(it.t + tpc, tiles_per_plane);
  };
  auto advance = [&](Item& it) {
    if (++it.t == it.t_end) {
      it.q += gridDim.x;
      if (it.q < num_chunks) first_tile(it);
    }
  };
  // the x halo of a tile reaches outside the image (same answer for every thread)
  auto at_edge = [&](const Item& it) {
    int ty0, tx0;
    tile_origin(it.t, ty0, tx0);
    return ty0 - G::R < 0 || ty0 + kFilterTileH + G::R > H || tx0 - G::RP < 0 ||
           tx0 + kTileW + G::RP > W;
  };
  auto stage = [&](const Item& it, int sb) {
    const int plane = (int)fdiv((uint32_t)it.q, fcpp);
    int ty0, tx0;
    tile_origin(it.t, ty0, tx0);
    T* sx = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES);
    T* sdy = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES + S::DY_OFF);
    if (use_tma) {
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bars + sb, (uint32_t)(S::X_BYTES + S::DY_BYTES));
        tma_load_3d(sx, &tmx, tx0 - G::RP, ty0 - G::R, plane, bars + sb);
        tma_load_3d(sdy, &tmdy, tx0, ty0, plane, bars + sb);
      }
    } else {
      const int64_t off = (int64_t)plane * H * W;
      stage_tile<T, G::R, G::RP, G::SP, S::NT, false>(sx, x + off, H, W, ty0, tx0, S::X_ROWS,
                                                      clamp != 0, vec != 0);
      stage_tile<T, 0, 0, kTileW, S::NT, false>(sdy, dy + off, H, W, ty0, tx0, kFilterTileH,
                                                false, vec != 0);
    }
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < S::NS; ++i) mbar_init(bars + i, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  cta_barrier();

  Item pf{(int)blockIdx.x, 0, 0};
  if (pf.q >= num_chunks) return;
  first_tile(pf);
  Item cs = pf;
  uint32_t phase = 0;    // bit s: parity of the next TMA completion on stage s
  uint32_t pending = 0;  // bit s: a TMA load into stage s is in flight
  // prologue: the first NS - 1 items (one commit group per item, empty past the end)
#pragma unroll
  for (int i = 0; i < S::NS - 1; ++i) {
    if (pf.q < num_chunks) {
      if (use_tma) pending |= 1u << i;
      stage(pf, i);
      advance(pf);
    }
    cp_async_commit();
  }

  float acc[S::AT][K];
#pragma unroll
  for (int s = 0; s < S::AT; ++s)
#pragma unroll
    for (int b = 0; b < K; ++b) acc[s][b] = 0.f;

  for (int sb = 0; cs.q < num_chunks; sb = (sb + 1 == S::NS) ? 0 : sb + 1) {
    // refill the stage released at the end of the previous item
    if (pf.q < num_chunks) {
      const int ps = sb == 0 ? S::NS - 1 : sb - 1;
      if (use_tma) pending |= 1u << ps;
      stage(pf, ps);
      advance(pf);
    }
    cp_async_commit();
    cp_async_wait_group<S::NS - 1>();  // the current item's cp.async copies have landed
    if (pending & (1u << sb)) {
      if (!mbar_wait(bars + sb, (phase >> sb) & 1u)) {
        record_error(err, kDevErrTimeout);
        *s_abort = 1;
      }
      phase ^= 1u << sb;
      pending &= ~(1u << sb);
    }
    cta_barrier();
    if (*s_abort) break;
    T* sx = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES);
    const T* sdy = reinterpret_cast<const T*>(sm + sb * S::STAGE_BYTES + S::DY_OFF);
    if (use_tma && clamp && at_edge(cs)) {
      int ty0, tx0;
      tile_origin(cs.t, ty0, tx0);
      clamp_fix<T, G::SP, S::NT>(sx, H, W, ty0, tx0, G::R, G::RP, S::X_ROWS);
    }
    dw_rows<K, S::AT, S::GT, kTileW, S::DR, T>(sdy + part * S::ROWS * kTileW + 4 * lane,
                                               sx + (part * S::ROWS + a_lo) * G::SP + 4 * lane,
                                               S::ROWS / S::DR, nrows, acc);
    const bool chunk_end = cs.t + 1 == cs.t_end;
    if (chunk_end) {
#pragma unroll
      for (int s = 0; s < S::AT; ++s)
#pragma unroll
        for (int b = 0; b < K; ++b) {
          float v = acc[s][b];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) sm_red[(warp * S::AT + s) * K + b] = v;
          acc[s][b] = 0.f;
        }
    }
    cta_barrier();  // stage sb is free again; sm_red is complete
    if (chunk_end) {
      for (int k = threadIdx.x; k < K * K; k += S::NT) {
        const int a = k / K, b = k - (k / K) * K;
        int gg = 0;
        while (gg + 1 < S::GT && group_lo(gg + 1, K, S::GT) <= a) ++gg;
        const int s = a - group_lo(gg, K, S::GT);
        float sum = 0.f;
        for (int p = 0; p < S::WPG; ++p) sum += sm_red[((gg * S::WPG + p) * S::AT + s) * K + b];
        partials[(int64_t)cs.q * K * K + k] = sum;
      }
      // sm_red is rewritten no earlier than the next chunk end, after another barrier
    }
    advance(cs);
  }
  cp_async_wait_group<0>();
  // after an abort: let the TMA loads still in flight land (bounded) before exiting
  for (int s = 0; s < S::NS; ++s)
    if (pending & (1u << s)) mbar_wait(bars + s, (phase >> s) & 1u);
}

// ------------------------------------------- backward with a staging ring
// Both gradients from one staged (x, dy) pair of halo tiles, like
// dw_bwd_kernel (warps 0-3: the input gradient g, warps 4-7: the filter
// gradient), but persistent over chunks of `tpc` consecutive tiles (chunk q
// runs on CTA q mod gridDim.x, the layout of dw_filter_kernel, so the same
// FP64 finalisation applies) with NS shared-memory stages: the copies of the
// tile NS - 1 items ahead are in flight while the current one is computed,
// across chunk boundaries too.  One CTA per SM.  It suits the HBM-bound small
// filters, whose single-stage fused kernel leaves its tile loads exposed; a
// tuning candidate for every K.  Tiles stay in the storage type (BF16 rows
// are widened as they enter registers).  The rotated filter of a chunk's
// channel goes to one of two buffers (chunk parity), written by the g warps.
template <int K, typename T>
struct RingShape {
  using G = Geo<K, sizeof(T)>;
  static constexpr int NT = kThreads;
  static constexpr int GT = dw_groups<K>();
  static constexpr int WPG = 4 / GT;
  static constexpr int AT = (K + GT - 1) / GT;
  static constexpr int DW_ROWS = kBwdTileH / WPG;
  static constexpr int BR = bwd_block_rows<K>();
  static constexpr int ROWS = kBwdTileH + 2 * G::R;
  static constexpr int T_BYTES = round_up(ROWS * G::SP * (int)sizeof(T), 128);
  static constexpr int STAGE_BYTES = 2 * T_BYTES;  // x, then dy (both with the halo)
  // three stages where they fit (two tiles in flight while one is computed)
  static constexpr int NS = 3 * STAGE_BYTES + 2 * Geo<K>::WPAD * 4 + 4 * AT * K * 4 + 64 <=
                                    227 * 1024
                                ? 3
                                : 2;
  static constexpr int SM_W = NS * STAGE_BYTES;
  static constexpr int SM_RED = SM_W + 2 * Geo<K>::WPAD * 4;
  static constexpr int SM_BAR = round_up(SM_RED + 4 * AT * K * 4, 8);
  static constexpr int SM_BYTES = SM_BAR + NS * 8 + 8;
  static_assert(DW_ROWS % BR == 0 && 16 % BR == 0, "whole row blocks");
  static_assert(SM_BYTES <= 227 * 1024, "shared memory");
};

template <typename T, int K>
__global__ void __launch_bounds__(kThreads, 1)
    dw_bwd_ring_kernel(const __grid_constant__ CUtensorMap tmx,
                       const __grid_constant__ CUtensorMap tmdy, const T* __restrict__ x,
                       const T* __restrict__ dy, const float* __restrict__ w, T* __restrict__ dx,
                       float* __restrict__ partials, int C, int H, int W, FastDiv ftx,
                       int tiles_per_plane, FastDiv fcpp, int tpc, int num_chunks, int clamp,
                       int vec, int use_tma, int* err) {
  using G = Geo<K, sizeof(T)>;
  using S = RingShape<K, T>;
  constexpr int KP = Geo<K>::KP;
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  float* sm_red = reinterpret_cast<float*>(sm + S::SM_RED);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::SM_BAR);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + S::SM_BAR + S::NS * 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool dw_warp = warp >= 4;
  const int wl = warp & 3;
  const int g = wl % S::GT, part = wl / S::GT;
  const int a_lo = group_lo(g, K, S::GT);
  const int nrows = group_lo(g + 1, K, S::GT) - a_lo;

  struct Item {
    int q;
    int t, t_end;
  };
  auto tile_origin = [&](int t, int& ty0, int& tx0) {
    const uint32_t r = fdiv((uint32_t)t, ftx);
    ty0 = (int)r * kBwdTileH;
    tx0 = (t - (int)(r * ftx.d)) * kTileW;
  };
  auto first_tile = [&](Item& it) {
    const int ch = it.q - (int)(fdiv((uint32_t)it.q, fcpp) * fcpp.d);
    it.t = ch * tpc;
    it.t_end = min(it.t + tpc, tiles_per_plane);
  };
  auto advance = [&](Item& it) {
    if (++it.t == it.t_end) {
      it.q += gridDim.x;
      if (it.q < num_chunks) first_tile(it);
    }
  };
  auto stage = [&](const Item& it, int sb) {
    const int plane = (int)fdiv((uint32_t)it.q, fcpp);
    int ty0, tx0;
    tile_origin(it.t, ty0, tx0);
    T* sx = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES);
    T* sdy = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES + S::T_BYTES);
    if (use_tma) {
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bars + sb, (uint32_t)(2 * S::ROWS * G::SP * (int)sizeof(T)));
        tma_load_3d(sx, &tmx, tx0 - G::RP, ty0 - G::R, plane, bars + sb);
        tma_load_3d(sdy, &tmdy, tx0 - G::RP, ty0 - G::R, plane, bars + sb);
      }
    } else {
      const int64_t off = (int64_t)plane * H * W;
      stage_tile<T, G::R, G::RP, G::SP, S::NT, false>(sx, x + off, H, W, ty0, tx0, S::ROWS,
                                                      clamp != 0, vec != 0);
      stage_tile<T, G::R, G::RP, G::SP, S::NT, false>(sdy, dy + off, H, W, ty0, tx0, S::ROWS,
                                                      false, vec != 0);
    }
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < S::NS; ++i) mbar_init(bars + i, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  cta_barrier();

  Item pf{(int)blockIdx.x, 0, 0};
  if (pf.q >= num_chunks) return;
  first_tile(pf);
  Item cs = pf;
  uint32_t phase = 0;    // bit s: parity of the next TMA completion on stage s
  uint32_t pending = 0;  // bit s: a TMA load into stage s is in flight
#pragma unroll
  for (int i = 0; i < S::NS - 1; ++i) {
    if (pf.q < num_chunks) {
      if (use_tma) pending |= 1u << i;
      stage(pf, i);
      advance(pf);
    }
    cp_async_commit();
  }

  float acc[S::AT][K];
#pragma unroll
  for (int s = 0; s < S::AT; ++s)
#pragma unroll
    for (int b = 0; b < K; ++b) acc[s][b] = 0.f;
  int nchunk = 0;  // chunks this CTA has finished (filter buffer parity)
  bool chunk_start = true;

  for (int sb = 0; cs.q < num_chunks; sb = (sb + 1 == S::NS) ? 0 : sb + 1) {
    // refill the stage released at the end of the previous item
    if (pf.q < num_chunks) {
      const int ps = sb == 0 ? S::NS - 1 : sb - 1;
      if (use_tma) pending |= 1u << ps;
      stage(pf, ps);
      advance(pf);
    }
    cp_async_commit();
    const int plane = (int)fdiv((uint32_t)cs.q, fcpp);
    float* swf = reinterpret_cast<float*>(sm + S::SM_W) + (nchunk & 1) * Geo<K>::WPAD;
    if (!dw_warp && chunk_start) {
      // the rotated filter of this chunk's channel; the other buffer may still
      // be read by the previous chunk's last tile
      const float* wc = w + (int64_t)(plane % C) * K * K;
      for (int k = threadIdx.x; k < K * KP; k += 128) {
        const int a = k / KP, b = k - (k / KP) * KP;
        swf[k] = b < K ? wc[(K - 1 - a) * K + (K - 1 - b)] : 0.f;
      }
    }
    cp_async_wait_group<S::NS - 1>();  // the current item's cp.async copies have landed
    if (pending & (1u << sb)) {
      if (!mbar_wait(bars + sb, (phase >> sb) & 1u)) {
        record_error(err, kDevErrTimeout);
        *s_abort = 1;
      }
      phase ^= 1u << sb;
      pending &= ~(1u << sb);
    }
    cta_barrier();
    if (*s_abort) break;
    T* sx = reinterpret_cast<T*>(sm + sb * S::STAGE_BYTES);
    const T* sdy = reinterpret_cast<const T*>(sm + sb * S::STAGE_BYTES + S::T_BYTES);
    int ty0, tx0;
    tile_origin(cs.t, ty0, tx0);
    if (use_tma && clamp &&
        (ty0 - G::R < 0 || ty0 + kBwdTileH + G::R > H || tx0 - G::RP < 0 ||
         tx0 + kTileW + G::RP > W))
      clamp_fix<T, G::SP, S::NT>(sx, H, W, ty0, tx0, G::R, G::RP, S::ROWS);
    if (!dw_warp) {
#pragma unroll 1
      for (int pass = 0; pass < 16 / S::BR; ++pass) {
        const int r0 = wl * 16 + pass * S::BR;
        float o[S::BR][4];
        fwd_block<K, S::BR, T>(sdy + r0 * G::SP + 4 * lane, swf, o);
        store_block<T, S::BR>(dx + (int64_t)plane * H * W, H, W, ty0 + r0, tx0 + 4 * lane,
                              vec != 0, o);
      }
    } else {
      const int r0 = part * S::DW_ROWS;
      dw_rows<K, S::AT, S::GT, G::SP, S::BR, T>(sdy + (r0 + G::R) * G::SP + G::RP + 4 * lane,
                                                sx + (r0 + a_lo) * G::SP + 4 * lane,
                                                S::DW_ROWS / S::BR, nrows, acc);
    }
    const bool chunk_end = cs.t + 1 == cs.t_end;
    if (chunk_end && dw_warp) {
#pragma unroll
      for (int s = 0; s < S::AT; ++s)
#pragma unroll
        for (int b = 0; b < K; ++b) {
          float v = acc[s][b];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) sm_red[(wl * S::AT + s) * K + b] = v;
          acc[s][b] = 0.f;
        }
    }
    cta_barrier();  // stage sb is free again; sm_red is complete
    if (chunk_end) {
      for (int k = threadIdx.x; k < K * K; k += S::NT) {
        const int a = k / K, b = k - (k / K) * K;
        int gg = 0;
        while (gg + 1 < S::GT && group_lo(gg + 1, K, S::GT) <= a) ++gg;
        const int s = a - group_lo(gg, K, S::GT);
        float sum = 0.f;
        for (int p = 0; p < S::WPG; ++p) sum += sm_red[((p * S::GT + gg) * S::AT + s) * K + b];
        partials[(int64_t)cs.q * K * K + k] = sum;
      }
      ++nchunk;
      // sm_red is rewritten no earlier than the next chunk end, after another barrier
    }
    chunk_start = chunk_end;
    advance(cs);
  }
  cp_async_wait_group<0>();
  // after an abort: let the TMA loads still in flight land (bounded) before exiting
  for (int s = 0; s < S::NS; ++s)
    if (pending & (1u << s)) mbar_wait(bars + s, (phase >> s) & 1u);
}

}  // namespace giga
