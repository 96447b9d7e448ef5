// up_batched.cu -- the sharpening benchmark (upsample, then filter; GigaAPI
// paper, Section 6.6) over a ragged "database" of images in ONE launch, the
// batch processing the paper set out to do and dropped (Section 5, "No Batch
// Processing for Images").
//
// Every image has its own size, channel count, integer scale s >= 2, filter
// size K <= 15 and filters w[C][K][K]; the output of an image is its
// upsampled grid (H*s) x (W*s) filtered with the border rule on that grid.
//
// Work: the host orders the images by filter size (largest first), then by
// tile count, and numbers their output tiles (64 x 128 pixels of one channel,
// channel-major) in that order.  Each filter size present in the batch is one
// launch of a kernel compiled for that size (at most 8 launches, whatever the
// number of images: 4 for a batch with K in {3, 5, 9, 11}); its CTA b runs
// the class's tile b, finding the image by a binary search over the table.
// Blocks start roughly in index order, so larger images go first and smaller
// ones fill the tail.  One kernel per size keeps each size's own register
// allocation and its filter taps in uniform registers; a single kernel
// switching on K per tile measured 125 registers instead of at most 72.  The
// 3 x 3 class is numbered in the polyphase kernel's items instead (plane,
// group of 8 input rows, 32 or 64 input columns) and run by persistent warps.  The
// per-tile and per-item bodies are the single-image kernels' (upsample.cuh),
// so every output equals that of giga_upsample_conv2d_fwd on the image alone,
// bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "upsample.cuh"

namespace giga {

constexpr int kUpRagMaxK = 15;
constexpr int kUpRagClasses = (kUpRagMaxK + 1) / 2;  // K = 15, 13, ..., 1

struct UpRagImage {
  const void* x;
  void* y;
  const float* w;
  int tile_base;  // number of this image's first tile
  int H, W, C, K, Ho, Wo;
  int tiles_x, tiles_y, n_tiles;  // n_tiles = C * tiles_x * tiles_y (K = 3: polyphase items)
  int vec;
  FastDiv fs;
  int mode;       // K = 3: the polyphase compilation (up3_mode)
  FastDiv fcb;    // K = 3: 32-column blocks per row group
  FastDiv fpp;    // K = 3: items per plane
};

// One launch: the images img_lo..img_hi of one filter size, whose tiles are
// numbered from tile0 on.
struct UpRagParams {
  const UpRagImage* images;
  int img_lo, img_hi, tile0;
  int clamp;
};

// One tile per CTA: CTA b runs tile tile0 + b, a tile of an image with filter
// size K.  Shared memory as in the single-image kernel (one stage).
template <typename T, int K>
__device__ __forceinline__ void up_rag_body(const UpRagParams& p) {
  using U = UpShape<K>;
  using G = Geo<K>;
  extern __shared__ __align__(16) float smem[];
  float* sx = smem;
  int* scol = reinterpret_cast<int*>(sx + U::EXP);
  int* rowoff = scol + G::SP;
  float* sw = reinterpret_cast<float*>(scol) + U::TABLES;
  float* ss = sw + round_up(G::WPAD, 4);
  const int tb = p.tile0 + (int)blockIdx.x;
  // the image: the last one of the class whose first tile is <= tb
  int lo = p.img_lo, hi = p.img_hi;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.images[mid].tile_base <= tb) lo = mid;
    else hi = mid - 1;
  }
  const UpRagImage& im = p.images[lo];
  const int t = tb - im.tile_base;
  const int per_plane = im.tiles_x * im.tiles_y;
  const int plane = t / per_plane;
  const int rr = t - plane * per_plane;
  const int ty = rr / im.tiles_x;
  const int ty0 = ty * U::TH, tx0 = (rr - ty * im.tiles_x) * kTileW;
  // input window: upsampled rows [ty0 - r, ty0 + 64 + r), columns
  // [tx0 - RP, tx0 + 128 + RP), clamped to the upsampled image, divided by s
  const int u_lo = max(ty0 - G::R, 0), u_hi = min(ty0 + U::TH + G::R, im.Ho) - 1;
  const int v_lo = max(tx0 - G::RP, 0), v_hi = min(tx0 + kTileW + G::RP, im.Wo) - 1;
  const int su0 = (int)fdiv((uint32_t)u_lo, im.fs), sv0 = (int)fdiv((uint32_t)v_lo, im.fs);
  const int nr = (int)fdiv((uint32_t)u_hi, im.fs) - su0 + 1;  // <= UpShape<K>::SRC_ROWS
  const int nc = (int)fdiv((uint32_t)v_hi, im.fs) - sv0 + 1;  // <= UpShape<K>::SRC_COLS
  stage_filter_async<K>(sw, im.w + (int64_t)plane * K * K, false, kThreads);
  const T* xp = static_cast<const T*>(im.x) + (int64_t)plane * im.H * im.W +
                (int64_t)su0 * im.W + sv0;
  up_stage_pixels<T, U::SRC_ROWS * U::SRC_COLS>(ss, U::SRC_COLS, xp, im.W, nr, nc);
  cp_async_commit();
  for (int k = threadIdx.x; k < G::SP; k += kThreads) sx[U::ZERO_OFF + k] = 0.f;
  cp_async_wait_group<0>();
  up_tile<T, K>(sx, U::ZERO_OFF, scol, rowoff, sw, ss, U::SRC_COLS, ty0, tx0, su0, sv0, nr, im.Ho,
                im.Wo, im.fs, p.clamp != 0, static_cast<T*>(im.y) + (int64_t)plane * im.Ho * im.Wo,
                im.vec != 0);
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) up_rag_kernel(UpRagParams p) {
  up_rag_body<T, K>(p);
}

// The 3 x 3 class: persistent warps over its polyphase items (an image's items
// contiguous, plane-major), the image found by a binary search, the summed
// taps recomputed when the (image, plane) changes.
constexpr int kUp3RagWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kUp3RagWarps * 32, 2) up3_rag_kernel(UpRagParams p, int n_items) {
  float wt[36];
  int img_cur = -1;
  uint32_t plane_cur = 0;
  for (int item = blockIdx.x * kUp3RagWarps + (threadIdx.x >> 5); item < n_items;
       item += gridDim.x * kUp3RagWarps) {
    const int tb = p.tile0 + item;
    int lo = p.img_lo, hi = p.img_hi;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.images[mid].tile_base <= tb) lo = mid;
      else hi = mid - 1;
    }
    const UpRagImage& im = p.images[lo];
    const uint32_t t = (uint32_t)(tb - im.tile_base);
    const uint32_t plane = fdiv(t, im.fpp);
    const uint32_t r = t - plane * im.fpp.d;
    const uint32_t rg = fdiv(r, im.fcb);
    const int cb = (int)(r - rg * im.fcb.d);
    if (lo != img_cur || plane != plane_cur) {
      up3_weights<0>(im.w + (int64_t)plane * 9, wt);
      img_cur = lo;
      plane_cur = plane;
    }
    const int sc = (int)im.fs.d;
    up3_item_mode<T>(im.mode, static_cast<const T*>(im.x) + (int64_t)plane * im.H * im.W,
                     static_cast<T*>(im.y) + (int64_t)plane * im.Ho * im.Wo, im.H, im.W, sc,
                     (int)rg * kUp3Rows, cb, p.clamp, wt);
  }
}

}  // namespace giga

using namespace giga;

struct giga_upsample_batched_plan_s {
  std::vector<UpRagImage> table;  // in processing order
  int border = 0, dtype = 0;
  int n_tiles = 0;
  int class_end[kUpRagClasses] = {};
  int img_end[kUpRagClasses] = {};
  size_t ws_bytes = 0;
  void* pinned = nullptr;
  cudaEvent_t uploaded = nullptr;
  const void* uploaded_ws = nullptr;  // the workspace the table went to
  bool pending = false;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// check_ptrs = false for size queries (shapes only).
giga_status_t build_up_plan(const giga_up_image_t* images, int32_t n, int32_t border,
                            int32_t dtype, bool check_ptrs, giga_upsample_batched_plan_s* plan) {
  if (n < 0 || (n > 0 && !images)) return fail(GIGA_ERR_INVALID_ARG, "bad image list");
  if (border != GIGA_BORDER_ZERO && border != GIGA_BORDER_CLAMP)
    return fail(GIGA_ERR_INVALID_ARG, "unknown border");
  if (dtype != GIGA_F32 && dtype != GIGA_BF16) return fail(GIGA_ERR_INVALID_ARG, "unknown dtype");
  plan->border = border;
  plan->dtype = dtype;
  const uintptr_t es = dtype == GIGA_BF16 ? 2 : 4;
  std::vector<UpRagImage> all;
  std::vector<int64_t> cost;
  for (int i = 0; i < n; ++i) {
    const giga_up_image_t& g = images[i];
    const std::string where = "image " + std::to_string(i) + ": ";
    if (g.H < 0 || g.W < 0 || g.C < 0) return fail(GIGA_ERR_INVALID_ARG, where + "negative dimension");
    if (g.K < 1 || g.K % 2 == 0 || g.K > 31)
      return fail(GIGA_ERR_INVALID_ARG, where + "K must be odd, 1..31");
    if (g.K > kUpRagMaxK)
      return fail(GIGA_ERR_UNSUPPORTED, where + "K above 15 in a batched upsample-then-filter");
    if (g.reserved != 0) return fail(GIGA_ERR_INVALID_ARG, where + "reserved must be 0");
    if (g.scale < 1) return fail(GIGA_ERR_INVALID_ARG, where + "scale must be >= 1");
    if (g.scale == 1)
      return fail(GIGA_ERR_UNSUPPORTED,
                  where + "scale 1 is the plain filter: use giga_conv2d_batched");
    const int64_t Ho = (int64_t)g.H * g.scale, Wo = (int64_t)g.W * g.scale;
    if (Ho >= (1LL << 31) || Wo >= (1LL << 31))
      return fail(GIGA_ERR_INVALID_ARG, where + "upsampled image too large");
    const int64_t n_in = (int64_t)g.C * g.H * g.W, n_out = (int64_t)g.C * Ho * Wo;
    if (n_out == 0) continue;
    if (check_ptrs) {
      if (!g.x || !g.y || !g.w) return fail(GIGA_ERR_INVALID_ARG, where + "NULL pointer");
      if (reinterpret_cast<uintptr_t>(g.x) % es || reinterpret_cast<uintptr_t>(g.y) % es ||
          reinterpret_cast<uintptr_t>(g.w) % 4)
        return fail(GIGA_ERR_MISALIGNED, where + "pointer not aligned to its element");
      if (overlaps(g.x, (size_t)n_in * es, g.y, (size_t)n_out * es))
        return fail(GIGA_ERR_INVALID_ARG, where + "y aliases x");
    }
    UpRagImage r;
    std::memset(&r, 0, sizeof(r));
    r.x = g.x;
    r.y = g.y;
    r.w = g.w;
    r.H = g.H;
    r.W = g.W;
    r.C = g.C;
    r.K = g.K;
    r.Ho = (int)Ho;
    r.Wo = (int)Wo;
    r.tiles_x = (int)((Wo + kTileW - 1) / kTileW);
    r.tiles_y = (int)((Ho + UpShape<1>::TH - 1) / UpShape<1>::TH);
    int64_t tiles = (int64_t)g.C * r.tiles_x * r.tiles_y;
    if (g.K == 3) {  // polyphase items: (plane, group of kUp3Rows rows, block of columns)
      r.mode = up3_mode(g.scale, g.y, (int)es, g.W);
      const int cols = up3_cols(r.mode);
      const int64_t rgs = (g.H + kUp3Rows - 1) / kUp3Rows, cbs = ((int64_t)g.W + cols - 1) / cols;
      tiles = (int64_t)g.C * rgs * cbs;
      r.fcb = make_fastdiv((uint32_t)cbs);
      r.fpp = make_fastdiv((uint32_t)(rgs * cbs));
    }
    if (tiles >= (1LL << 31)) return fail(GIGA_ERR_INVALID_ARG, where + "too many tiles");
    r.n_tiles = (int)tiles;
    const uintptr_t va = dtype == GIGA_F32 ? 16 : 8;
    r.vec = (Wo % 4 == 0 && reinterpret_cast<uintptr_t>(g.y) % va == 0) ? 1 : 0;
    r.fs = make_fastdiv((uint32_t)g.scale);
    all.push_back(r);
    cost.push_back(tiles);
  }
  // Longest first: the largest filters (cost K^2 per pixel), larger images
  // first among equals; an image's tiles stay contiguous.
  std::vector<int> order(all.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (all[a].K != all[b].K) return all[a].K > all[b].K;
    return cost[a] > cost[b];
  });
  int64_t tiles = 0;
  plan->table.clear();
  for (int i : order) {
    UpRagImage r = all[i];
    r.tile_base = (int)tiles;
    tiles += r.n_tiles;
    if (tiles >= (1LL << 31)) return fail(GIGA_ERR_INVALID_ARG, "batch too large for one launch");
    plan->table.push_back(r);
  }
  plan->n_tiles = (int)tiles;
  // class c (K = 15 - 2c): tiles before class_end[c], images before img_end[c]
  for (int c = 0, i = 0; c < kUpRagClasses; ++c) {
    while (i < (int)plan->table.size() && plan->table[i].K == kUpRagMaxK - 2 * c) ++i;
    plan->img_end[c] = i;
    plan->class_end[c] = i < (int)plan->table.size() ? plan->table[i].tile_base : (int)tiles;
  }
  plan->ws_bytes = align256(std::max<size_t>(sizeof(UpRagImage) * plan->table.size(), 1));
  return GIGA_OK;
}

giga_status_t check_up_ws(const giga_upsample_batched_plan_s* plan, void* ws, size_t ws_bytes) {
  if (!ws) return fail(GIGA_ERR_WORKSPACE, "workspace is NULL");
  if (ws_bytes < plan->ws_bytes)
    return fail(GIGA_ERR_WORKSPACE, "workspace too small, need " + std::to_string(plan->ws_bytes));
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return fail(GIGA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  return GIGA_OK;
}

template <typename T, int K>
cudaError_t up_rag_launch_k(const UpRagParams& p, int n_tiles, cudaStream_t st) {
  const size_t smem = (size_t)UpShape<K>::SM_FLOATS_1 * 4;
  cudaError_t e;
  if ((e = set_smem_once<up_rag_kernel<T, K>>(smem)) != cudaSuccess) return e;
  up_rag_kernel<T, K><<<n_tiles, kThreads, smem, st>>>(p);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t up3_rag_launch(const UpRagParams& p, int n_items, cudaStream_t st) {
  static int ctas_per_sm[64] = {};  // per device, measured at its first launch
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int n = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, up3_rag_kernel<T>, kUp3RagWarps * 32, 0);
    if (e != cudaSuccess) return e;
    per_sm = n > 0 ? n : 1;
  }
  const int grid = (int)std::min<int64_t>((n_items + kUp3RagWarps - 1) / kUp3RagWarps,
                                          (int64_t)per_sm * sm_count());
  up3_rag_kernel<T><<<grid, kUp3RagWarps * 32, 0, st>>>(p, n_items);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t up_rag_launch(int K, const UpRagParams& p, int n_tiles, cudaStream_t st) {
  switch (K) {
    case 1: return up_rag_launch_k<T, 1>(p, n_tiles, st);
    case 3: return up3_rag_launch<T>(p, n_tiles, st);
    case 5: return up_rag_launch_k<T, 5>(p, n_tiles, st);
    case 7: return up_rag_launch_k<T, 7>(p, n_tiles, st);
    case 9: return up_rag_launch_k<T, 9>(p, n_tiles, st);
    case 11: return up_rag_launch_k<T, 11>(p, n_tiles, st);
    case 13: return up_rag_launch_k<T, 13>(p, n_tiles, st);
    case 15: return up_rag_launch_k<T, 15>(p, n_tiles, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

extern "C" {

giga_status_t giga_upsample_batched_plan_create(const giga_up_image_t* images, int32_t n,
                                                int32_t border, int32_t dtype,
                                                giga_upsample_batched_plan_t* plan) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  auto* p = new (std::nothrow) giga_upsample_batched_plan_s();
  if (!p) return fail(GIGA_ERR_INVALID_ARG, "out of host memory");
  giga_status_t s = build_up_plan(images, n, border, dtype, true, p);
  if (s != GIGA_OK) {
    delete p;
    return s;
  }
  *plan = p;
  return GIGA_OK;
}

giga_status_t giga_upsample_batched_plan_workspace_size(giga_upsample_batched_plan_t plan,
                                                        size_t* bytes) {
  clear_error();
  if (!plan || !bytes) return fail(GIGA_ERR_INVALID_ARG, "NULL argument");
  *bytes = plan->ws_bytes;
  return GIGA_OK;
}

giga_status_t giga_upsample_batched_plan_upload(giga_upsample_batched_plan_t plan, void* ws,
                                                size_t ws_bytes, void* stream) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  giga_status_t s = check_up_ws(plan, ws, ws_bytes);
  if (s != GIGA_OK) return s;
  if (plan->table.empty()) return GIGA_OK;  // nothing to launch
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(UpRagImage) * plan->table.size();
  cudaError_t e;
  if (plan->pending) {  // a previous upload may still read the pinned buffer
    if ((e = cudaEventSynchronize(plan->uploaded)) != cudaSuccess) return cuda_fail(e, "upload wait");
    plan->pending = false;
  }
  if (!plan->pinned) {
    if ((e = cudaMallocHost(&plan->pinned, bytes)) != cudaSuccess) return cuda_fail(e, "pinned table");
    std::memcpy(plan->pinned, plan->table.data(), bytes);
  }
  if (!plan->uploaded && (e = cudaEventCreateWithFlags(&plan->uploaded, cudaEventDisableTiming)))
    return cuda_fail(e, "event");
  if ((e = cudaMemcpyAsync(ws, plan->pinned, bytes, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "table upload");
  if ((e = cudaEventRecord(plan->uploaded, st))) return cuda_fail(e, "event record");
  plan->pending = true;
  plan->uploaded_ws = ws;
  return GIGA_OK;
}

giga_status_t giga_upsample_batched_plan_run(giga_upsample_batched_plan_t plan, void* ws,
                                             size_t ws_bytes, void* stream) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  giga_status_t s = check_up_ws(plan, ws, ws_bytes);
  if (s != GIGA_OK) return s;
  if (plan->table.empty()) return GIGA_OK;
  if (!plan->uploaded) return fail(GIGA_ERR_INVALID_ARG, "plan was never uploaded");
  if (ws != plan->uploaded_ws)
    return fail(GIGA_ERR_WORKSPACE, "run with the workspace the table was uploaded to");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  UpRagParams p;
  p.images = static_cast<const UpRagImage*>(ws);
  p.clamp = plan->border == GIGA_BORDER_CLAMP;
  for (int c = 0; c < kUpRagClasses; ++c) {
    const int img_lo = c == 0 ? 0 : plan->img_end[c - 1];
    const int tile0 = c == 0 ? 0 : plan->class_end[c - 1];
    const int n_tiles = plan->class_end[c] - tile0;
    if (n_tiles == 0) continue;
    p.img_lo = img_lo;
    p.img_hi = plan->img_end[c] - 1;
    p.tile0 = tile0;
    const int K = kUpRagMaxK - 2 * c;
    cudaError_t e = plan->dtype == GIGA_F32 ? up_rag_launch<float>(K, p, n_tiles, st)
                                            : up_rag_launch<__nv_bfloat16>(K, p, n_tiles, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched upsample-then-filter launch");
  }
  return GIGA_OK;
}

void giga_upsample_batched_plan_destroy(giga_upsample_batched_plan_t plan) {
  if (!plan) return;
  if (plan->pending) cudaEventSynchronize(plan->uploaded);
  if (plan->uploaded) cudaEventDestroy(plan->uploaded);
  if (plan->pinned) cudaFreeHost(plan->pinned);
  delete plan;
}

giga_status_t giga_upsample_conv2d_batched(const giga_up_image_t* images, int32_t n,
                                           int32_t border, int32_t dtype, void* ws,
                                           size_t ws_bytes, void* stream) {
  clear_error();
  giga_upsample_batched_plan_t plan = nullptr;
  giga_status_t s = giga_upsample_batched_plan_create(images, n, border, dtype, &plan);
  if (s != GIGA_OK) return s;
  s = giga_upsample_batched_plan_upload(plan, ws, ws_bytes, stream);
  if (s == GIGA_OK) s = giga_upsample_batched_plan_run(plan, ws, ws_bytes, stream);
  std::string detail = giga_last_error_detail();
  giga_upsample_batched_plan_destroy(plan);
  if (s != GIGA_OK) fail(s, detail);
  return s;
}

giga_status_t giga_upsample_conv2d_batched_workspace_size(const giga_up_image_t* images,
                                                          int32_t n, size_t* bytes) {
  clear_error();
  if (!bytes) return fail(GIGA_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  giga_upsample_batched_plan_s plan;
  giga_status_t s = build_up_plan(images, n, GIGA_BORDER_ZERO, GIGA_F32, false, &plan);
  if (s != GIGA_OK) return s;
  *bytes = plan.ws_bytes;
  return GIGA_OK;
}

}  // extern "C"
