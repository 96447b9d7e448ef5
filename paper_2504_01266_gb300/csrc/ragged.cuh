// ragged.cuh -- one persistent launch over a ragged batch of images (different
// sizes and filter sizes), driven by a tile table in device memory.
//
// The GigaAPI paper wanted to process a "database" of images in one go and
// gave up (Section 5, "No Batch Processing for Images"); this kernel does it:
//  * the host cuts every (image, channel) into chunks of up to 4 tiles of
//    64 x 128 pixels (1 to 32, powers of 2: the plan's autotuner times them) and
//    sorts the chunks longest first (cost K^2 per pixel);
//  * CTAs (one per SM, 16 warps) pull chunk numbers from an atomic counter,
//    stage each tile's x and dy once, and run the three ops on it with fixed
//    warp roles: warps 0-3 forward, 4-7 input gradient, 8-15 filter gradient.
//    The filter gradient's per-pixel work equals each other role's, but its
//    inner loop reaches a lower FMA rate; for K >= 11 all 8 of its warps work
//    (in groups of at most 3 filter rows, so the union of the filter-size
//    bodies fits the 128 registers a thread of a 16-warp CTA has) and the
//    three roles finish a tile at about the same time; for K <= 9, where the
//    forward and input-gradient roles bound the tile, 4 of them work (the
//    other 4 stage and synchronise only: 8 working warps measured no faster);
//  * each chunk writes one K*K vector of FP32 filter-gradient partials; the
//    CTA that completes the last chunk of an (image, channel) -- detected with
//    a per-(image, channel) atomic counter after a memory fence -- sums that
//    image-channel's partials in FP64 in chunk order (deterministic) and, for
//    the clamp border, folds the edges of dx.  No CTA ever waits for another.
#pragma once

#include "dw_fold.cuh"
#include "dw_kernels.cuh"

namespace giga {

constexpr int kRagThreads = 512;
constexpr int kRagDwWarps = 8;  // filter-gradient warps (warps 8-15)
constexpr int kRagTilesPerChunk = 4;  // the plan's default; the autotuner may pick 1 to 32
constexpr int kRagMaxK = 15;

struct RagImage {
  const void* x;
  void* y;
  const void* dy;
  void* dx;
  const float* w;
  float* dw;
  int64_t partial_base;  // float offset of this image's partials
  int H, W, C, K;
  int nch;      // chunks per channel
  int ic_base;  // completion counter of (this image, channel 0)
  int vec;
  int pad;
};

struct RagChunk {
  int image, channel, tile_begin, tile_end;
};

struct RagParams {
  const RagImage* images;
  const RagChunk* chunks;
  int* counters;  // [0]: work counter, [1 + ic]: finished chunks of (image, channel) ic
  float* partials;
  int n_chunks;
  int tpc;  // tiles per chunk
  int ops;  // GIGA_OP_* bitmask
  int border;
};

// Filter-row groups of the 8 filter-gradient warps for K >= 11: fewer rows
// per warp keep the accumulators within the 128 registers a thread of a
// 16-warp CTA has (K = 11: 4 groups of at most 3 rows; K >= 13: 8 groups of
// at most 2 rows, one warp each).
template <int K>
constexpr int rag_groups() {
  return K <= 7 ? 1 : (K <= 9 ? 2 : (K <= 11 ? 4 : 8));
}
// filter-gradient warps that work for this K (the others only stage and sync)
template <int K>
constexpr int rag_dw_active() {
  return K <= 9 ? 4 : 8;
}

template <int K, typename T>
struct RagShape {
  using G = Geo<K, sizeof(T)>;
  static constexpr int GT = K <= 9 ? dw_groups<K>() : rag_groups<K>();
  static constexpr int WPG = rag_dw_active<K>() / GT;
  static constexpr int AT = (K + GT - 1) / GT;
  static constexpr int DW_ROWS = kBwdTileH / WPG;
  static constexpr int ROWS = kBwdTileH + 2 * G::R;
};

// Shared memory, sized for the largest filter: two tile stages (x and dy
// tiles), two filter buffers (a chunk's filter and its rotation; indexed by
// chunk parity so the next chunk's filter can be staged while the current one
// is in use), the filter-gradient reduction rows and two ints.
template <typename T>
struct RagLayout {
  using G = Geo<kRagMaxK, sizeof(T)>;
  static constexpr int TILE = round_up((kBwdTileH + 2 * G::R) * G::SP * (int)sizeof(T), 128);
  static constexpr int STAGE = 2 * TILE;          // x, then dy
  static constexpr int WB = G::WPAD * 4;          // one filter
  static constexpr int FILT = 2 * STAGE;          // [2][w, wf]
  static constexpr int RED = FILT + 4 * WB;       // [2 chunks][w, wf] filters
  static constexpr int RED_FLOATS = 66;           // K = 11: 6 rows x 11 taps
  static constexpr int INTS = RED + kRagDwWarps * RED_FLOATS * 4;
  static constexpr int SM_BYTES = INTS + 16;
  static_assert(RagShape<11, T>::AT * 11 <= RED_FLOATS && RagShape<15, T>::AT * 15 <= RED_FLOATS,
                "reduction rows");
  static_assert(SM_BYTES <= 227 * 1024, "shared memory");
};

template <typename T>
constexpr size_t rag_max_smem() {
  return (size_t)RagLayout<T>::SM_BYTES;
}

// Issue the copies of tile t of chunk ch (image im) into stage sb and, for the
// first tile of a chunk, its filters into filter buffer fb (no commit).
template <typename T>
__device__ __forceinline__ void rag_stage(const RagParams& p, const RagChunk& ch,
                                          const RagImage& im, int t, char* sm, int sb, int fb,
                                          bool filters) {
  using L = RagLayout<T>;
  const int K = im.K, R = (K - 1) / 2, RP = geo_rp(K, sizeof(T)), SP = kTileW + 2 * RP;
  const int H = im.H, W = im.W;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
  const int64_t off = (int64_t)ch.channel * H * W;
  const bool do_fwd = p.ops & 1, do_dx = p.ops & 2, do_dw = p.ops & 4;
  const bool clamp = p.border == 1, vec = im.vec != 0;
  T* sx = reinterpret_cast<T*>(sm + sb * L::STAGE);
  T* sdy = reinterpret_cast<T*>(sm + sb * L::STAGE + L::TILE);
  if (do_fwd || do_dw)
    stage_tile_rt<T, kRagThreads>(sx, static_cast<const T*>(im.x) + off, H, W, ty0, tx0,
                                  kBwdTileH + 2 * R, R, RP, SP, clamp, vec);
  if (do_dx || do_dw)
    stage_tile_rt<T, kRagThreads>(sdy, static_cast<const T*>(im.dy) + off, H, W, ty0, tx0,
                                  kBwdTileH + 2 * R, R, RP, SP, false, vec);
  // w may be NULL when neither the forward nor the input gradient is requested
  if (filters && (do_fwd || do_dx)) {
    const float* wc = im.w + (int64_t)ch.channel * K * K;
    float* f = reinterpret_cast<float*>(sm + L::FILT + fb * 2 * L::WB);
    stage_filter_rt<kRagThreads>(f, wc, K, false);
    stage_filter_rt<kRagThreads>(f + L::WB / 4, wc, K, true);
  }
}

// One chunk: its first tile is already in stage sb (copies in flight), its
// filters in filter buffer fb.  While tile t is computed, the copies of the
// next tile -- the next of this chunk, or the first of chunk `cn` -- go to
// the other stage.  Returns the stage holding the next chunk's first tile.
template <typename T, int K>
__device__ __forceinline__ int rag_chunk(const RagParams& p, const RagChunk& ch,
                                         const RagImage& im, int cn, char* sm, int sb, int fb,
                                         int* s_flag) {
  using G = Geo<K, sizeof(T)>;
  using S = RagShape<K, T>;
  using L = RagLayout<T>;
  constexpr int KK = K * K;
  float* sm_red = reinterpret_cast<float*>(sm + L::RED);
  const float* sm_w = reinterpret_cast<const float*>(sm + L::FILT + fb * 2 * L::WB);
  const float* sm_wf = sm_w + L::WB / 4;

  const int H = im.H, W = im.W;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int64_t off = (int64_t)ch.channel * H * W;
  const bool do_fwd = p.ops & 1, do_dx = p.ops & 2, do_dw = p.ops & 4;
  const bool clamp = p.border == 1, vec = im.vec != 0;
  T* yp = do_fwd ? static_cast<T*>(im.y) + off : nullptr;
  T* dxp = do_dx ? static_cast<T*>(im.dx) + off : nullptr;
  const float* wc = (do_fwd || do_dx) ? im.w + (int64_t)ch.channel * KK : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int role = warp < 8 ? warp >> 2 : 2, wl = warp < 8 ? (warp & 3) : warp - 8;
  const int g = wl % S::GT;
  const int part = wl / S::GT;
  const int a_lo = group_lo(g, K, S::GT);
  const int nrows = group_lo(g + 1, K, S::GT) - a_lo;
  float acc[S::AT][K];
#pragma unroll
  for (int s = 0; s < S::AT; ++s)
#pragma unroll
    for (int b = 0; b < K; ++b) acc[s][b] = 0.f;

  for (int t = ch.tile_begin; t < ch.tile_end; ++t) {
    if (t + 1 < ch.tile_end) {
      rag_stage<T>(p, ch, im, t + 1, sm, sb ^ 1, fb, false);
    } else if (cn < p.n_chunks) {
      const RagChunk chn = p.chunks[cn];
      const RagImage imn = p.images[chn.image];
      rag_stage<T>(p, chn, imn, chn.tile_begin, sm, sb ^ 1, fb ^ 1, true);
    }
    cp_async_commit();
    cp_async_wait_group<1>();  // this tile's copies (committed one tile earlier) have landed
    cta_barrier();
    const T* sx = reinterpret_cast<const T*>(sm + sb * L::STAGE);
    const T* sdy = reinterpret_cast<const T*>(sm + sb * L::STAGE + L::TILE);
    const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
    if (role < 2) {
      if (role == 0 ? do_fwd : do_dx) {
        const T* src = role == 0 ? sx : sdy;
        const float* f = role == 0 ? sm_w : sm_wf;
        T* dst = role == 0 ? yp : dxp;
        constexpr int BR = bwd_block_rows<K>();
#pragma unroll 1
        for (int pass = 0; pass < 16 / BR; ++pass) {
          const int r0 = wl * 16 + pass * BR;
          float o[BR][4];
          fwd_block<K, BR, T>(src + r0 * G::SP + 4 * lane, f, o);
          store_block<T, BR>(dst, H, W, ty0 + r0, tx0 + 4 * lane, vec, o);
        }
      }
    } else if (do_dw && wl < rag_dw_active<K>()) {
      constexpr int BR = bwd_block_rows<K>();
      const int r0 = part * S::DW_ROWS;
      dw_rows<K, S::AT, S::GT, G::SP, BR, T>(sdy + (r0 + G::R) * G::SP + G::RP + 4 * lane,
                                             sx + (r0 + a_lo) * G::SP + 4 * lane,
                                             S::DW_ROWS / BR, nrows, acc);
    }
    cta_barrier();  // stage sb is free for the copies two tiles ahead
    sb ^= 1;
  }

  // filter-gradient partial of this chunk: warp butterflies, then a fixed-order
  // sum over the group's warps
  if (role == 2 && do_dw && wl < rag_dw_active<K>()) {
#pragma unroll
    for (int s = 0; s < S::AT; ++s)
#pragma unroll
      for (int b = 0; b < K; ++b) {
        float v = acc[s][b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm_red[wl * L::RED_FLOATS + s * K + b] = v;
      }
  }
  cta_barrier();
  const int ic = im.ic_base + ch.channel;
  float* part_c = p.partials + im.partial_base + (int64_t)ch.channel * im.nch * KK;
  if (do_dw) {
    const int j = ch.tile_begin / p.tpc;
    for (int k = threadIdx.x; k < KK; k += kRagThreads) {
      const int a = k / K, b = k - (k / K) * K;
      int gg = 0;
      while (gg + 1 < S::GT && group_lo(gg + 1, K, S::GT) <= a) ++gg;
      const int s = a - group_lo(gg, K, S::GT);
      float sum = 0.f;
      for (int q = 0; q < S::WPG; ++q) sum += sm_red[(q * S::GT + gg) * L::RED_FLOATS + s * K + b];
      part_c[(int64_t)j * KK + k] = sum;
    }
  }
  if (do_dw || (do_dx && clamp)) {
    __threadfence();
    cta_barrier();
    if (threadIdx.x == 0) *s_flag = atomicAdd(p.counters + 1 + ic, 1) == im.nch - 1;
    cta_barrier();
    if (*s_flag) {
      __threadfence();
      if (do_dw) {
        for (int k = threadIdx.x; k < KK; k += kRagThreads) {
          double s = 0.0;
          for (int j = 0; j < im.nch; ++j) s += (double)__ldcg(part_c + (int64_t)j * KK + k);
          im.dw[(int64_t)ch.channel * KK + k] = (float)s;
        }
      }
      if (do_dx && clamp) {
        const int64_t edges = edge_pixels(H, W);
        const T* gsrc = static_cast<const T*>(im.dy) + off;
        for (int64_t e = threadIdx.x; e < edges; e += kRagThreads)
          fold_edge_pixel<T>(gsrc, wc, dxp, H, W, K, e);
      }
    }
  }
  cta_barrier();  // sm_red and s_flag are reused by the next chunk
  return sb;
}

template <typename T>
__global__ void __launch_bounds__(kRagThreads, 1) rag_kernel(RagParams p) {
  extern __shared__ __align__(128) float smem[];
  using L = RagLayout<T>;
  char* sm = reinterpret_cast<char*>(smem);
  volatile int* s_next = reinterpret_cast<volatile int*>(sm + L::INTS);
  int* s_flag = reinterpret_cast<int*>(sm + L::INTS + 4);
  if (threadIdx.x == 0) *s_next = atomicAdd(p.counters, 1);
  cta_barrier();
  int c = *s_next;
  if (c >= p.n_chunks) return;
  int sb = 0, fb = 0;
  {
    const RagChunk ch = p.chunks[c];
    const RagImage im = p.images[ch.image];
    rag_stage<T>(p, ch, im, ch.tile_begin, sm, sb, fb, true);
    cp_async_commit();
  }
  for (;;) {
    cta_barrier();  // every thread has read the previous *s_next
    if (threadIdx.x == 0) *s_next = atomicAdd(p.counters, 1);  // one chunk ahead
    cta_barrier();
    const int cn = *s_next;
    const RagChunk ch = p.chunks[c];
    const RagImage im = p.images[ch.image];
    switch (im.K) {
      case 1: sb = rag_chunk<T, 1>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 3: sb = rag_chunk<T, 3>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 5: sb = rag_chunk<T, 5>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 7: sb = rag_chunk<T, 7>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 9: sb = rag_chunk<T, 9>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 11: sb = rag_chunk<T, 11>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      case 13: sb = rag_chunk<T, 13>(p, ch, im, cn, sm, sb, fb, s_flag); break;
      default: sb = rag_chunk<T, 15>(p, ch, im, cn, sm, sb, fb, s_flag); break;
    }
    if (cn >= p.n_chunks) break;
    c = cn;
    fb ^= 1;
  }
  cp_async_wait_group<0>();
}

cudaError_t rag_launch_f32(const RagParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t rag_launch_bf16(const RagParams& p, int grid, size_t smem, cudaStream_t st);

}  // namespace giga
