// upsample.cuh -- pieces shared by the single-image and the batched
// upsample-then-filter kernels (upsample.cu, up_batched.cu): the tile
// geometry and per-tile body of the general K x K pass, and the polyphase
// body of the 3 x 3 pass.
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
// One item, one warp: 32 consecutive input columns x kUp3Rows input rows of one
// plane, a 3 x 3 register window over the rows (side neighbours by warp
// shuffle).  Each lane writes the s x s output block of its input pixel, row
// by row, with CE-element vector stores (s % CE == 0 and y aligned to CE
// elements).  S is s when compiled for one scale (2, 4, 8), else 0.
constexpr int kUp3Rows = 8;

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

// One output row of a lane's PX input pixels: for pixel p, vl[p], then s - 2
// times vm[p], then vr[p] (S: s when known at compile time, else 0).  Either
// CE = PX * S (one store for all pixels) or CE divides s; dst is aligned to
// CE elements.
template <typename T, int CE, int S, int PX>
__device__ __forceinline__ void up3_row(T* dst, int s, const float (&vl)[PX],
                                        const float (&vm)[PX], const float (&vr)[PX]) {
  if constexpr (S != 0 && CE > S) {
    static_assert(CE == PX * S, "one store covers every pixel of the lane");
    float e[CE];
#pragma unroll
    for (int k = 0; k < CE; ++k) {
      const int q = k / S, v = k % S;
      e[k] = v == 0 ? vl[q] : (v == S - 1 ? vr[q] : vm[q]);
    }
    Up3Store<T, CE>::put(dst, e);
  } else {
    const int n = S ? S : s;
#pragma unroll
    for (int p = 0; p < PX; ++p)
#pragma unroll
      for (int v0 = 0; v0 < (S ? S : n); v0 += CE) {
        float e[CE];
#pragma unroll
        for (int k = 0; k < CE; ++k) {
          const int v = v0 + k;
          e[k] = v == 0 ? vl[p] : (v == n - 1 ? vr[p] : vm[p]);
        }
        Up3Store<T, CE>::put(dst + p * n + v0, e);
      }
  }
}

// s = 2 has no middle row or column class.
template <int S>
__host__ __device__ constexpr bool up3_used(int R) { return S != 2 || R != 1; }

// Wt[R][C][i][j] of one channel (wc: its 3 x 3 taps): the taps of the row
// slot i of class R and the column slot j of class C, summed row-major.
template <int S>
__device__ __forceinline__ void up3_weights(const float* __restrict__ wc, float (&wt)[36]) {
  float tap[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) tap[k] = __ldg(wc + k);
#pragma unroll
  for (int R = 0; R < 3; ++R)
#pragma unroll
    for (int C = 0; C < 3; ++C)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float sum = 0.f;
          if (up3_used<S>(R) && up3_used<S>(C)) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b)
                if ((up3_taps(R, i) >> a & 1) && (up3_taps(C, j) >> b & 1)) sum += tap[a * 3 + b];
          }
          wt[((R * 3 + C) * 2 + i) * 2 + j] = sum;
        }
}

// One item: input rows i0 .. i0 + kUp3Rows - 1 (those below H) and columns
// 32 PX cb .. 32 PX cb + 32 PX - 1 (PX consecutive ones per lane) of the
// plane xp (H x W), output plane yp (H s x W s).  Every lane of the warp calls
// it.
template <typename T, int CE, int S, int PX>
__device__ __forceinline__ void up3_item(const T* __restrict__ xp, T* __restrict__ yp, int H,
                                         int W, int s, int i0, int cb, int clamp,
                                         const float (&wt)[36]) {
  if (S) s = S;
  const int lane = threadIdx.x & 31;
  const int J0 = (cb * 32 + lane) * PX;  // the lane's first input column
  const int64_t Wo = (int64_t)W * s;
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
  // Columns J0 - 1 .. J0 + PX of every input row the item needs (its rows and
  // the halo above and below), all loads issued before the first use.  Lanes
  // past W hold the border value of their columns, which is what their left
  // neighbour needs.
  constexpr int NR = kUp3Rows + 2;
  const int side_col = lane == 0 ? J0 - 1 : J0 + PX;  // the neighbour outside the warp
  float cm[NR][PX], cs[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
#pragma unroll
    for (int p = 0; p < PX; ++p) cm[k][p] = ld(i0 - 1 + k, J0 + p);
    cs[k] = (lane == 0 || lane == 31) ? ld(i0 - 1 + k, side_col) : 0.f;
  }
  float cl[NR], cr[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const float up = __shfl_up_sync(0xffffffffu, cm[k][PX - 1], 1);
    const float dn = __shfl_down_sync(0xffffffffu, cm[k][0], 1);
    cl[k] = lane == 0 ? cs[k] : up;
    cr[k] = lane == 31 ? cs[k] : dn;
  }
  // column c of the lane's window: J0 - 1 + c, c in [0, PX + 2)
  auto col = [&](int k, int c) { return c == 0 ? cl[k] : (c == PX + 1 ? cr[k] : cm[k][c - 1]); };
  // the output blocks of input pixels (i0, J0 ..), then one block row down per row
  T* o = yp + (int64_t)i0 * s * Wo + (int64_t)J0 * s;
#pragma unroll
  for (int k = 0; k < kUp3Rows; ++k, o += s * Wo) {
    if (i0 + k >= H) break;
    float v[3][3][PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      const float n[3][3] = {{col(k, p), col(k, p + 1), col(k, p + 2)},
                             {col(k + 1, p), col(k + 1, p + 1), col(k + 1, p + 2)},
                             {col(k + 2, p), col(k + 2, p + 1), col(k + 2, p + 2)}};
#pragma unroll
      for (int R = 0; R < 3; ++R)
#pragma unroll
        for (int C = 0; C < 3; ++C) {
          float acc = 0.f;
          bool started = false;
          if (up3_used<S>(R) && up3_used<S>(C)) {
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
          }
          v[R][C][p] = acc;
        }
    }
    if (J0 + PX <= W) {
      up3_row<T, CE, S, PX>(o, s, v[0][0], v[0][1], v[0][2]);
#pragma unroll
      for (int u = 1; u < (S ? S - 1 : s - 1); ++u)
        up3_row<T, CE, S, PX>(o + u * Wo, s, v[1][0], v[1][1], v[1][2]);
      up3_row<T, CE, S, PX>(o + (s - 1) * Wo, s, v[2][0], v[2][1], v[2][2]);
    } else if constexpr (PX > 1) {
      // the last pixels of a row: element stores for those inside the image
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        if (J0 + p >= W) break;
        for (int u = 0; u < s; ++u) {
          const int R = u == 0 ? 0 : (u == s - 1 ? 2 : 1);
          for (int q = 0; q < s; ++q) {
            const int C = q == 0 ? 0 : (q == s - 1 ? 2 : 1);
            Elem<T>::store(o + u * Wo + p * s + q, v[R][C][p]);
          }
        }
      }
    }
  }
}

// The compilation of the polyphase body for scale s, output address y and
// input width W: s itself where compiled for it (2, 4, 8), else run-time s,
// with the widest stores s, y's alignment and W allow (at most 32 bytes).
// Modes 0, 1: s = 2, 4 with two input pixels per lane (one store of 2 s
// elements per output row; W even keeps every output row aligned); 2-4:
// (CE, S) = (2, 2), (4, 4), (8, 8); 5: one 32-byte sector, run-time s; 6: 8
// elements (BF16 only); 7: 4; 8: 2; 9: 1.
inline int up3_mode(int s, const void* y, int elem_bytes, int64_t W) {
  const uintptr_t yp = reinterpret_cast<uintptr_t>(y);
  auto fits = [&](int ce) { return s % ce == 0 && yp % (uintptr_t)(ce * elem_bytes) == 0; };
  auto pair_fits = [&](int ce) { return W % 2 == 0 && yp % (uintptr_t)(ce * elem_bytes) == 0; };
  if (s == 2 && pair_fits(4)) return 0;
  if (s == 4 && pair_fits(8) && 8 * elem_bytes <= 32) return 1;
  if (s == 2 && fits(2)) return 2;
  if (s == 4 && fits(4)) return 3;
  if (s == 8 && fits(8)) return 4;
  if (fits(32 / elem_bytes)) return 5;
  if (elem_bytes == 2 && fits(8)) return 6;
  if (fits(4)) return 7;
  if (fits(2)) return 8;
  return 9;
}

// Input columns per item of mode m.
__host__ __device__ constexpr int up3_cols(int m) { return m <= 1 ? 64 : 32; }

// The body of mode m (a warp-uniform switch).
template <typename T>
__device__ __forceinline__ void up3_item_mode(int m, const T* __restrict__ xp, T* __restrict__ yp,
                                              int H, int W, int s, int i0, int cb, int clamp,
                                              const float (&wt)[36]) {
  constexpr int kSector = 32 / (int)sizeof(T);
  switch (m) {
    case 0: up3_item<T, 4, 2, 2>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 1: up3_item<T, 8, 4, 2>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 2: up3_item<T, 2, 2, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 3: up3_item<T, 4, 4, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 4: up3_item<T, 8, 8, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 5: up3_item<T, kSector, 0, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 6:
      if constexpr (sizeof(T) == 2) up3_item<T, 8, 0, 1>(xp, yp, H, W, s, i0, cb, clamp, wt);
      break;
    case 7: up3_item<T, 4, 0, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    case 8: up3_item<T, 2, 0, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
    default: up3_item<T, 1, 0, 1>(xp, yp, H, W, s, i0, cb, clamp, wt); break;
  }
}

}  // namespace giga
