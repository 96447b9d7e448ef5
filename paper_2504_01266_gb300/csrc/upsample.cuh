// upsample.cuh -- pieces shared by the single-image and the batched
// upsample-then-filter kernels (upsample.cu, up_batched.cu): fixed-divisor
// division, the tile geometry and the per-tile body.
//
//   up[p][q] = x[p / s][q / s]                                   (integer division)
//   y[p][q]  = sum_{a,b} w[a][b] * up~[p + a - r][q + b - r]     (GigaAPI paper,
//              Sections 4.2.3 and 4.2.4, run back to back as in Section 6.6)
//
// up~ applies the border rule on the (H*s) x (W*s) upsampled image.
#pragma once

#include "dw_kernels.cuh"

namespace giga {

// Geometry of one 64 x 128 output tile of the upsampled grid (8 warps, 8 rows
// each) for a K x K filter and a scale s >= 2: the staged input pixels under
// the tile's window, the same rows expanded along the columns of the FP32 halo
// tile (plus one row of zeros), and the tables that map halo rows and columns
// to them.
template <int K>
struct UpShape {
  using G = Geo<K>;
  static constexpr int TH = kWarps * 8;
  static constexpr int ROWS = TH + 2 * G::R;                   // halo rows
  static constexpr int SRC_ROWS = ROWS / 2 + 2;                // input rows under the window (s >= 2)
  static constexpr int SRC_COLS = round_up(G::SP / 2 + 2, 4);  // input columns (pitch)
  static constexpr int STAGE = round_up(G::WPAD, 4) + SRC_ROWS * SRC_COLS;  // filter + pixels
  static constexpr int EXP = (SRC_ROWS + 1) * G::SP;           // expanded rows + the zero row
  static constexpr int ZERO_OFF = SRC_ROWS * G::SP;            // float offset of the zero row
  static constexpr int TABLES = G::SP + round_up(ROWS, 4);     // column map, row offsets
  static constexpr int SM_FLOATS_1 = EXP + TABLES + STAGE;     // one tile per CTA
  static constexpr int SM_FLOATS = SM_FLOATS_1 + STAGE;        // two stages
};

// Copy the nr x nc input pixels of a tile's window (rows from src, row
// stride W) to ss (pitch `pitch`), every copy in flight at once: FP32 by
// 4-byte cp.async, BF16 by loads issued before the widened stores.  No
// commit.  The (row, column) of a thread's k-th element advances by a
// constant step, so there is one division per tile.
template <typename T, int MAXN>
__device__ __forceinline__ void up_stage_pixels(float* __restrict__ ss, int pitch,
                                                const T* __restrict__ src, int64_t W, int nr,
                                                int nc) {
  const int n = nr * nc;
  int r = threadIdx.x / nc, c = threadIdx.x - (threadIdx.x / nc) * nc;
  const int dr = kThreads / nc, dc = kThreads - dr * nc;
  if constexpr (sizeof(T) == 4) {
    for (int k = threadIdx.x; k < n; k += kThreads) {
      cp_async4(ss + r * pitch + c, src + r * W + c, true);
      r += dr;
      c += dc;
      if (c >= nc) {
        c -= nc;
        ++r;
      }
    }
  } else {
    constexpr int PER = (MAXN + kThreads - 1) / kThreads;
    float v[PER];
    int rr[PER], cc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      rr[i] = r;
      cc[i] = c;
      if (i * kThreads + (int)threadIdx.x < n) v[i] = Elem<T>::load(src + r * W + c);
      r += dr;
      c += dc;
      if (c >= nc) {
        c -= nc;
        ++r;
      }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i)
      if (i * kThreads + (int)threadIdx.x < n) ss[rr[i] * pitch + cc[i]] = v[i];
  }
}

// fwd_group with the shared address of every input row taken from a table:
// input row ir of the group starts at base + rowoff[ir].
template <int K, int PY, int A>
__device__ __forceinline__ void fwd_group_tab(const float* __restrict__ base,
                                              const int* __restrict__ rowoff,
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
    load_window_row<K, float>(base + rowoff[ir], buf);
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

// acc[py][px] = sum_{a,b} f[a*KP + b] * (row py + a of the table)[OFF + px + b]
template <int K, int PY>
__device__ __forceinline__ void fwd_block_tab(const float* __restrict__ base,
                                              const int* __restrict__ rowoff,
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
    fwd_group_tab<K, PY, A>(base, rowoff + g * A, f + g * A * Geo<K>::KP, acc);
  if constexpr (REM > 0)
    fwd_group_tab<K, PY, REM>(base, rowoff + NG * A, f + NG * A * Geo<K>::KP, acc);
}

// One output tile, after its nr input rows and its filter have been copied to
// shared memory (every thread has waited for its own copies): the input
// window starts at input row su0, column sv0 and is stored in ss with row
// pitch src_pitch; sw is the staged filter (rows padded to Geo<K>::KP).
//
// Halo cell (sr, sc) of the tile is upsampled pixel (u, v) = (ty0 - r + sr,
// tx0 - RP + sc) under the border rule on the upsampled image (zero: the cell
// is 0; clamp: (u, v) clamped), i.e. input pixel (u / s, v / s).  The column
// mapping is the same for every row (scol[sc]: the copied input column, -1
// for zero), so each copied input row is expanded once along the columns into
// sx (row e at e * SP); a halo row is then just a pointer: rowoff[sr] is the
// offset of its expanded input row, or zero_off, a row of zeros the caller
// keeps in sx, for rows outside the image under the zero border.  The forward
// loop reads its input rows through rowoff; its arithmetic and order are the
// depthwise forward's.  Ends with a barrier, after which sx, the tables and
// ss may be reused (the zero row is left as it was).
template <typename T, int K>
__device__ __forceinline__ void up_tile(float* __restrict__ sx, int zero_off,
                                        int* __restrict__ scol, int* __restrict__ rowoff,
                                        const float* __restrict__ sw,
                                        const float* __restrict__ ss, int src_pitch, int ty0,
                                        int tx0, int su0, int sv0, int nr, int Ho, int Wo,
                                        const FastDiv& fs, bool clamp, T* __restrict__ yplane,
                                        bool vec) {
  using G = Geo<K>;
  using U = UpShape<K>;
  constexpr int PY = 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int sc = threadIdx.x; sc < G::SP; sc += kThreads) {
    int v = tx0 - G::RP + sc;
    int m = -1;
    if (clamp || (v >= 0 && v < Wo)) {
      v = v < 0 ? 0 : (v >= Wo ? Wo - 1 : v);
      m = (int)fdiv((uint32_t)v, fs) - sv0;
    }
    scol[sc] = m;
  }
  for (int sr = threadIdx.x; sr < U::ROWS; sr += kThreads) {
    int u = ty0 - G::R + sr;
    int off = zero_off;
    if (clamp || (u >= 0 && u < Ho)) {
      u = u < 0 ? 0 : (u >= Ho ? Ho - 1 : u);
      off = ((int)fdiv((uint32_t)u, fs) - su0) * G::SP;
    }
    rowoff[sr] = off;
  }
  cta_barrier();  // copies of this tile landed; tables ready
  constexpr int CPR = G::SP / 4;
  for (int k = threadIdx.x; k < nr * CPR; k += kThreads) {
    const int e = k / CPR, sc = (k - (k / CPR) * CPR) * 4;
    const int4 m = *reinterpret_cast<const int4*>(scol + sc);
    const float* srow = ss + e * src_pitch;
    float4 v;
    v.x = m.x >= 0 ? srow[m.x] : 0.f;
    v.y = m.y >= 0 ? srow[m.y] : 0.f;
    v.z = m.z >= 0 ? srow[m.z] : 0.f;
    v.w = m.w >= 0 ? srow[m.w] : 0.f;
    *reinterpret_cast<float4*>(sx + e * G::SP + sc) = v;
  }
  cta_barrier();
  float acc[PY][4];
  fwd_block_tab<K, PY>(sx + 4 * lane, rowoff + warp * PY, sw, acc);
  store_block<T, PY>(yplane, Ho, Wo, ty0 + warp * PY, tx0 + 4 * lane, vec, acc);
  cta_barrier();  // the expanded rows, tables and the staged pixels are free again
}

}  // namespace giga
