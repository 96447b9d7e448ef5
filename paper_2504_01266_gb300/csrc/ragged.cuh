// ragged.cuh -- one persistent launch over a ragged batch of images (different
// sizes and filter sizes), driven by a tile table in device memory.
//
// The GigaAPI paper wanted to process a "database" of images in one go and
// gave up (Section 5, "No Batch Processing for Images"); this kernel does it:
//  * the host cuts every (image, channel) into chunks of up to 4 tiles of
//    64 x 128 pixels and sorts the chunks longest first (cost K^2 per pixel);
//  * CTAs (one per SM, 12 warps) pull chunk numbers from an atomic counter,
//    stage each tile's x and dy once, and run the three ops on it with fixed
//    warp roles: warps 0-3 forward, 4-7 input gradient, 8-11 filter gradient;
//  * each chunk writes one K*K vector of FP32 filter-gradient partials; the
//    CTA that completes the last chunk of an (image, channel) -- detected with
//    a per-(image, channel) atomic counter after a memory fence -- sums that
//    image-channel's partials in FP64 in chunk order (deterministic) and, for
//    the clamp border, folds the edges of dx.  No CTA ever waits for another.
#pragma once

#include "dw_fold.cuh"
#include "dw_kernels.cuh"

namespace giga {

constexpr int kRagThreads = 384;
constexpr int kRagTilesPerChunk = 4;
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
  int ops;  // GIGA_OP_* bitmask
  int border;
};

template <int K, typename T>
struct RagShape {
  using G = Geo<K, sizeof(T)>;
  static constexpr int GT = dw_groups<K>();
  static constexpr int WPG = 4 / GT;
  static constexpr int AT = (K + GT - 1) / GT;
  static constexpr int DW_ROWS = kBwdTileH / WPG;
  static constexpr int ROWS = kBwdTileH + 2 * G::R;
  // byte offsets: staged tiles in the storage type, filters and reduction FP32
  static constexpr int SM_X = 0;
  static constexpr int SM_DY = ROWS * G::SP * (int)sizeof(T);
  static constexpr int SM_W = 2 * ROWS * G::SP * (int)sizeof(T);
  static constexpr int SM_WF = SM_W + G::WPAD * 4;
  static constexpr int SM_RED = SM_WF + G::WPAD * 4;
  static constexpr int SM_BYTES = SM_RED + 4 * AT * K * 4;
};

template <typename T>
constexpr size_t rag_max_smem() {
  return (size_t)RagShape<15, T>::SM_BYTES;
}

template <typename T, int K>
__device__ __forceinline__ void rag_chunk(const RagParams& p, const RagChunk& ch,
                                          const RagImage& im, float* smem, int* s_flag) {
  using G = Geo<K, sizeof(T)>;
  using S = RagShape<K, T>;
  constexpr int KK = K * K;
  char* sm = reinterpret_cast<char*>(smem);
  T* sm_x = reinterpret_cast<T*>(sm + S::SM_X);
  T* sm_dy = reinterpret_cast<T*>(sm + S::SM_DY);
  float* sm_w = reinterpret_cast<float*>(sm + S::SM_W);
  float* sm_wf = reinterpret_cast<float*>(sm + S::SM_WF);
  float* sm_red = reinterpret_cast<float*>(sm + S::SM_RED);

  const int H = im.H, W = im.W;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int64_t off = (int64_t)ch.channel * H * W;
  const bool do_fwd = p.ops & 1, do_dx = p.ops & 2, do_dw = p.ops & 4;
  const bool need_x = do_fwd || do_dw, need_dy = do_dx || do_dw;
  const bool clamp = p.border == 1, vec = im.vec != 0;
  const T* xp = need_x ? static_cast<const T*>(im.x) + off : nullptr;
  const T* dyp = need_dy ? static_cast<const T*>(im.dy) + off : nullptr;
  T* yp = do_fwd ? static_cast<T*>(im.y) + off : nullptr;
  T* dxp = do_dx ? static_cast<T*>(im.dx) + off : nullptr;
  // w may be NULL when neither the forward nor the input gradient is requested
  const float* wc = (do_fwd || do_dx) ? im.w + (int64_t)ch.channel * KK : nullptr;
  if (wc) {
    stage_filter<K>(sm_w, wc, false, kRagThreads);
    stage_filter<K>(sm_wf, wc, true, kRagThreads);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int role = warp >> 2, wl = warp & 3;

  if (role < 2) {
    const bool active = role == 0 ? do_fwd : do_dx;
    const T* src = role == 0 ? sm_x : sm_dy;
    const float* f = role == 0 ? sm_w : sm_wf;
    T* dst = role == 0 ? yp : dxp;
    for (int t = ch.tile_begin; t < ch.tile_end; ++t) {
      const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
      cta_barrier();
      if (need_x)
        stage_tile<T, G::R, G::RP, G::SP, kRagThreads>(sm_x, xp, H, W, ty0, tx0, S::ROWS, clamp,
                                                       vec);
      if (need_dy)
        stage_tile<T, G::R, G::RP, G::SP, kRagThreads>(sm_dy, dyp, H, W, ty0, tx0, S::ROWS,
                                                       false, vec);
      stage_wait();
      if (active) {
        constexpr int BR = bwd_block_rows<K>();
#pragma unroll 1
        for (int pass = 0; pass < 16 / BR; ++pass) {
          const int r0 = wl * 16 + pass * BR;
          float acc[BR][4];
          fwd_block<K, BR, T>(src + r0 * G::SP + 4 * lane, f, acc);
          store_block<T, BR>(dst, H, W, ty0 + r0, tx0 + 4 * lane, vec, acc);
        }
      }
    }
    cta_barrier();
    cta_barrier();
  } else {
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
      const int ty0 = (t / tiles_x) * kBwdTileH, tx0 = (t % tiles_x) * kTileW;
      cta_barrier();
      if (need_x)
        stage_tile<T, G::R, G::RP, G::SP, kRagThreads>(sm_x, xp, H, W, ty0, tx0, S::ROWS, clamp,
                                                       vec);
      if (need_dy)
        stage_tile<T, G::R, G::RP, G::SP, kRagThreads>(sm_dy, dyp, H, W, ty0, tx0, S::ROWS,
                                                       false, vec);
      stage_wait();
      if (do_dw) {
        constexpr int BR = bwd_block_rows<K>();
        const int r0 = part * S::DW_ROWS;
        dw_rows<K, S::AT, S::GT, G::SP, BR, T>(sm_dy + (r0 + G::R) * G::SP + G::RP + 4 * lane,
                                               sm_x + (r0 + a_lo) * G::SP + 4 * lane,
                                               S::DW_ROWS / BR, nrows, acc);
      }
    }
    cta_barrier();
#pragma unroll
    for (int s = 0; s < S::AT; ++s)
#pragma unroll
      for (int b = 0; b < K; ++b) {
        float v = acc[s][b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm_red[(wl * S::AT + s) * K + b] = v;
      }
    cta_barrier();
  }

  const int ic = im.ic_base + ch.channel;
  float* part_c = p.partials + im.partial_base + (int64_t)ch.channel * im.nch * KK;
  if (do_dw) {
    const int j = ch.tile_begin / kRagTilesPerChunk;
    for (int k = threadIdx.x; k < KK; k += kRagThreads) {
      const int a = k / K, b = k - (k / K) * K;
      int g = 0;
      while (g + 1 < S::GT && group_lo(g + 1, K, S::GT) <= a) ++g;
      const int s = a - group_lo(g, K, S::GT);
      float sum = 0.f;
      for (int q = 0; q < S::WPG; ++q) sum += sm_red[((q * S::GT + g) * S::AT + s) * K + b];
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
        const T* g = static_cast<const T*>(im.dy) + off;
        for (int64_t e = threadIdx.x; e < edges; e += kRagThreads)
          fold_edge_pixel<T>(g, wc, dxp, H, W, K, e);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kRagThreads, 1) rag_kernel(RagParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_idx, s_flag;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(p.counters, 1);
    cta_barrier();
    const int idx = s_idx;
    if (idx >= p.n_chunks) break;
    const RagChunk ch = p.chunks[idx];
    const RagImage im = p.images[ch.image];
    switch (im.K) {
      case 1: rag_chunk<T, 1>(p, ch, im, smem, &s_flag); break;
      case 3: rag_chunk<T, 3>(p, ch, im, smem, &s_flag); break;
      case 5: rag_chunk<T, 5>(p, ch, im, smem, &s_flag); break;
      case 7: rag_chunk<T, 7>(p, ch, im, smem, &s_flag); break;
      case 9: rag_chunk<T, 9>(p, ch, im, smem, &s_flag); break;
      case 11: rag_chunk<T, 11>(p, ch, im, smem, &s_flag); break;
      case 13: rag_chunk<T, 13>(p, ch, im, smem, &s_flag); break;
      default: rag_chunk<T, 15>(p, ch, im, smem, &s_flag); break;
    }
    cta_barrier();
  }
}

cudaError_t rag_launch_f32(const RagParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t rag_launch_bf16(const RagParams& p, int grid, size_t smem, cudaStream_t st);

}  // namespace giga
