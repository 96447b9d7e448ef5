// upsample.cu -- nearest-neighbour upsampling by an integer factor s (the
// GigaAPI paper, Section 4.2.3) and the paper's sharpening benchmark fused
// into one pass (Section 6.6): the K x K depthwise filter applied to the
// upsampled image, whose pixels are read straight from the small input while
// a tile is staged, so the upsampled image never goes to HBM.
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

// ------------------------- upsample, then the 3 x 3 filter: polyphase form
// For K = 3 and s >= 2 the window of output pixel (s I + u, s J + v) covers
// the upsampled rows s I + u - 1 .. s I + u + 1, which are input rows I - 1
// and I when u = 0, row I alone when 0 < u < s - 1, rows I and I + 1 when
// u = s - 1 (columns likewise).  So
//   y[s I + u][s J + v] = sum_{i,j} Wt[R][C][i][j] * x~[I + o(R, i)][J + o(C, j)]
// with row class R = R(u) in {top, middle, bottom}, column class C = C(v) in
// {left, middle, right}, at most two input offsets o per class, and Wt the sum
// of the taps that land on the same input pixel: 1, 2 or 4 multiply-adds per
// output pixel instead of 9, no expanded rows, and all middle columns of a
// class row equal.  The border rule applies to x~ directly: floor(P / s)
// leaves [0, H) exactly when P leaves [0, H s), and the nearest upsampled
// pixel of a clamped row is that of the nearest input row.  Rounding differs
// from filtering the stored upsampled image (the taps of one input pixel are
// added before the multiply); the FP32 error stays within gamma(K^2 + 4) of
// the sum of |terms|.
//
// One warp: 32 consecutive input columns x kUp3Rows input rows, a 3 x 3
// register window sliding down the rows (side neighbours by warp shuffle); a
// CTA: kUp3Warps warps stacked vertically.  Each lane writes the s x s output
// block of its input pixel, row by row, with CE-element vector stores
// (s % CE == 0 and y aligned to CE elements).
constexpr int kUp3Rows = 8;
constexpr int kUp3Warps = 8;

// Class R (0: top / left, 1: middle, 2: bottom / right): the taps (bit a:
// tap a) that land on its input offset slot i, and that offset.
__host__ __device__ constexpr int up3_taps(int R, int i) {
  return R == 0 ? (i == 0 ? 1 : 6) : R == 1 ? (i == 0 ? 7 : 0) : (i == 0 ? 3 : 4);
}
__host__ __device__ constexpr int up3_off(int R, int i) {
  return R == 0 ? (i == 0 ? -1 : 0) : R == 1 ? 0 : (i == 0 ? 0 : 1);
}

template <typename T, int CE> struct Up3Store;
// 32-byte stores (sm_100 and later): one lane writes a whole sector.
__device__ __forceinline__ void st_global_v8(void* p, uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t a4, uint32_t a5, uint32_t a6,
                                             uint32_t a7) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a0),
               "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7)
               : "memory");
}

template <int CE> struct Up3Store<float, CE> {
  static __device__ __forceinline__ void put(float* p, const float (&e)[CE]) {
    if constexpr (CE == 8)
      st_global_v8(p, __float_as_uint(e[0]), __float_as_uint(e[1]), __float_as_uint(e[2]),
                   __float_as_uint(e[3]), __float_as_uint(e[4]), __float_as_uint(e[5]),
                   __float_as_uint(e[6]), __float_as_uint(e[7]));
    else if constexpr (CE == 4) *reinterpret_cast<float4*>(p) = make_float4(e[0], e[1], e[2], e[3]);
    else if constexpr (CE == 2) *reinterpret_cast<float2*>(p) = make_float2(e[0], e[1]);
    else *p = e[0];
  }
};
template <int CE> struct Up3Store<__nv_bfloat16, CE> {
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ void put(__nv_bfloat16* p, const float (&e)[CE]) {
    if constexpr (CE == 16)
      st_global_v8(p, pack(e[0], e[1]), pack(e[2], e[3]), pack(e[4], e[5]), pack(e[6], e[7]),
                   pack(e[8], e[9]), pack(e[10], e[11]), pack(e[12], e[13]), pack(e[14], e[15]));
    else if constexpr (CE == 8)
      *reinterpret_cast<uint4*>(p) =
          make_uint4(pack(e[0], e[1]), pack(e[2], e[3]), pack(e[4], e[5]), pack(e[6], e[7]));
    else if constexpr (CE == 4)
      *reinterpret_cast<uint2*>(p) = make_uint2(pack(e[0], e[1]), pack(e[2], e[3]));
    else if constexpr (CE == 2)
      *reinterpret_cast<uint32_t*>(p) = pack(e[0], e[1]);
    else
      *p = __float2bfloat16_rn(e[0]);
  }
};

// One output row of an input pixel's block: vl, then s - 2 times vm, then vr
// (S: s when known at compile time, else 0).
template <typename T, int CE, int S>
__device__ __forceinline__ void up3_row(T* dst, int s, float vl, float vm, float vr) {
  const int n = S ? S : s;
#pragma unroll
  for (int v0 = 0; v0 < (S ? S : n); v0 += CE) {
    float e[CE];
#pragma unroll
    for (int k = 0; k < CE; ++k) {
      const int v = v0 + k;
      e[k] = v == 0 ? vl : (v == n - 1 ? vr : vm);
    }
    Up3Store<T, CE>::put(dst + v0, e);
  }
}

template <typename T, int CE, int S>
__global__ void __launch_bounds__(kUp3Warps * 32) up3_poly_kernel(
    const T* __restrict__ x, const float* __restrict__ w, T* __restrict__ y, FastDiv fc, int H,
    int W, int s, FastDiv fcb, FastDiv frb, uint32_t items, int clamp) {
  if (S) s = S;  // the scale, a compile-time constant for S != 0
  const int lane = threadIdx.x & 31;
  const int64_t Wo = (int64_t)W * s;
  // s = 2 has no middle row or column class
  auto used = [](int R) { return S != 2 || R != 1; };
  float wt[36];  // Wt[R][C][i][j] of channel c_cur
  int c_cur = -1;
  // every warp on its own: items (plane, group of kUp3Rows input rows, block of
  // 32 input columns), the column block fastest
  for (uint32_t item = blockIdx.x * kUp3Warps + (threadIdx.x >> 5); item < items;
       item += gridDim.x * kUp3Warps) {
    const uint32_t q = fdiv(item, fcb);
    const int cb = (int)(item - q * fcb.d);
    const uint32_t plane = fdiv(q, frb);
    const int rg = (int)(q - plane * frb.d);
    const int c = (int)(plane - fdiv(plane, fc) * fc.d);
    const int i0 = rg * kUp3Rows;
    const int J = cb * 32 + lane;
    const T* xp = x + (int64_t)plane * H * W;
    // x~ with the border rule
    auto ld = [&](int r, int col) -> float {
      if (clamp) {
        r = min(max(r, 0), H - 1);
        col = min(max(col, 0), W - 1);
      } else if (r < 0 || r >= H || col < 0 || col >= W) {
        return 0.f;
      }
      return Elem<T>::load(xp + (int64_t)r * W + col);
    };
    // Columns J - 1, J, J + 1 of every input row the item needs (its rows and
    // the halo above and below), all loads issued before the first use.
    // Lanes past W hold the border value of their column, which is what
    // their left neighbour needs.
    constexpr int NR = kUp3Rows + 2;
    const int side_col = lane == 0 ? J - 1 : J + 1;  // the neighbour outside the warp
    float cm[NR], cs[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      cm[k] = ld(i0 - 1 + k, J);
      cs[k] = (lane == 0 || lane == 31) ? ld(i0 - 1 + k, side_col) : 0.f;
    }
    if (c != c_cur) {  // the summed taps of this channel
      float tap[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) tap[k] = __ldg(w + (int64_t)c * 9 + k);
#pragma unroll
      for (int R = 0; R < 3; ++R)
#pragma unroll
        for (int C = 0; C < 3; ++C)
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              if (!used(R) || !used(C)) continue;
              float sum = 0.f;
#pragma unroll
              for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
                for (int b2 = 0; b2 < 3; ++b2)
                  if ((up3_taps(R, i) >> a2 & 1) && (up3_taps(C, j) >> b2 & 1))
                    sum += tap[a2 * 3 + b2];
              wt[((R * 3 + C) * 2 + i) * 2 + j] = sum;
            }
      c_cur = c;
    }
    float cl[NR], cr[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const float up = __shfl_up_sync(0xffffffffu, cm[k], 1);
      const float dn = __shfl_down_sync(0xffffffffu, cm[k], 1);
      cl[k] = lane == 0 ? cs[k] : up;
      cr[k] = lane == 31 ? cs[k] : dn;
    }
    // the output block of input pixel (i0, J), then one block row down per row
    T* o = y + ((int64_t)plane * H + i0) * s * Wo + (int64_t)J * s;
#pragma unroll
    for (int k = 0; k < kUp3Rows; ++k, o += s * Wo) {
      if (i0 + k >= H) break;
      const float n[3][3] = {{cl[k], cm[k], cr[k]},
                             {cl[k + 1], cm[k + 1], cr[k + 1]},
                             {cl[k + 2], cm[k + 2], cr[k + 2]}};
      float v[3][3];
#pragma unroll
      for (int R = 0; R < 3; ++R)
#pragma unroll
        for (int C = 0; C < 3; ++C) {
          float acc = 0.f;
          bool started = false;
          if (!used(R) || !used(C)) {
            v[R][C] = 0.f;
            continue;
          }
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              if (up3_taps(R, i) == 0 || up3_taps(C, j) == 0) continue;
              const float t = wt[((R * 3 + C) * 2 + i) * 2 + j];
              const float xv = n[1 + up3_off(R, i)][1 + up3_off(C, j)];
              acc = started ? fmaf(t, xv, acc) : t * xv;
              started = true;
            }
          v[R][C] = acc;
        }
      if (J < W) {
        up3_row<T, CE, S>(o, s, v[0][0], v[0][1], v[0][2]);
#pragma unroll
        for (int u = 1; u < (S ? S - 1 : s - 1); ++u)
          up3_row<T, CE, S>(o + u * Wo, s, v[1][0], v[1][1], v[1][2]);
        up3_row<T, CE, S>(o + (s - 1) * Wo, s, v[2][0], v[2][1], v[2][2]);
      }
    }
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

template <typename T, int CE, int S>
static cudaError_t up3_launch_ce(const UpArgs& a, cudaStream_t st) {
  const int64_t rgs = (a.H + kUp3Rows - 1) / kUp3Rows;
  const int64_t cbs = (a.W + 31) / 32;
  const int64_t items = a.N * a.C * rgs * cbs;
  if (items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  static int ctas_per_sm[64] = {};  // per device, measured at its first launch
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, up3_poly_kernel<T, CE, S>, kUp3Warps * 32, 0);
    if (e != cudaSuccess) return e;
    per_sm = n > 0 ? n : 1;
  }
  const int64_t grid = std::min<int64_t>((items + kUp3Warps - 1) / kUp3Warps,
                                         (int64_t)per_sm * sm_count());
  up3_poly_kernel<T, CE, S><<<(unsigned)grid, kUp3Warps * 32, 0, st>>>(
      static_cast<const T*>(a.x), a.w, static_cast<T*>(a.y), make_fastdiv((uint32_t)a.C),
      (int)a.H, (int)a.W, a.s, make_fastdiv((uint32_t)cbs), make_fastdiv((uint32_t)rgs),
      (uint32_t)items, a.border);
  note_launch();
  return cudaGetLastError();
}

// K = 3: the polyphase kernel with the widest stores that s and y's alignment
// allow (at most 32 bytes: one sector per lane); scales 2, 4 and 8 compiled
// for their value (the class loops and stores unrolled), others at run time.
template <typename T>
static cudaError_t up3_launch(const UpArgs& a, cudaStream_t st) {
  const uintptr_t yp = reinterpret_cast<uintptr_t>(a.y);
  auto fits = [&](int ce) { return a.s % ce == 0 && yp % (ce * sizeof(T)) == 0; };
  constexpr int kSector = 32 / (int)sizeof(T);  // elements per 32-byte store
  if (a.s == 2 && fits(2)) return up3_launch_ce<T, 2, 2>(a, st);
  if (a.s == 4 && fits(4)) return up3_launch_ce<T, 4, 4>(a, st);
  if (a.s == 8 && fits(8)) return up3_launch_ce<T, 8, 8>(a, st);
  if (fits(kSector)) return up3_launch_ce<T, kSector, 0>(a, st);
  if (fits(8) && 8 < kSector) return up3_launch_ce<T, 8, 0>(a, st);
  if (fits(4)) return up3_launch_ce<T, 4, 0>(a, st);
  if (fits(2)) return up3_launch_ce<T, 2, 0>(a, st);
  return up3_launch_ce<T, 1, 0>(a, st);
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
