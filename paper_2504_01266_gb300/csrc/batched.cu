// batched.cu -- host side of the ragged batch: validation, the tile table
// (plan), workspace layout, upload and the persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "ragged.cuh"

using namespace giga;

struct giga_batched_plan_s {
  std::vector<giga_image_t> descs;  // the caller's descriptors (rebuilt per chunk size)
  std::vector<RagImage> images;
  std::vector<RagChunk> chunks;
  int tpc = kRagTilesPerChunk;      // tiles per chunk
  int uploaded_tpc = 0;             // tiles per chunk of the table last uploaded (0: none)
  const void* uploaded_ws = nullptr;  // the workspace that table went to
  std::vector<int> empty_filter_grads;  // images whose dw must be zeroed (no pixels)
  int ops = 0, border = 0, dtype = 0;
  int n_ic = 0;
  int max_k = 1;
  int64_t partial_floats = 0;
  size_t off_chunks = 0, off_counters = 0, off_partials = 0, ws_bytes = 0;
  size_t ws_max = 0, table_max = 0;  // over every tiles-per-chunk candidate (the smallest chunks)
  void* pinned = nullptr;
  size_t table_bytes = 0, pinned_bytes = 0;
  cudaEvent_t uploaded = nullptr;
  bool pending = false;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

giga_status_t validate_image(const giga_image_t& im, int i, int ops, int dtype) {
  const std::string where = "image " + std::to_string(i) + ": ";
  if (im.H < 0 || im.W < 0 || im.C < 0)
    return fail(GIGA_ERR_INVALID_ARG, where + "negative dimension");
  if (im.K < 1 || im.K > kRagMaxK || im.K % 2 == 0)
    return fail(im.K > kRagMaxK && im.K <= 31 && im.K % 2 ? GIGA_ERR_UNSUPPORTED
                                                           : GIGA_ERR_INVALID_ARG,
                where + "K must be odd and at most 15 in a ragged batch");
  const int64_t n = (int64_t)im.C * im.H * im.W;
  if (n == 0) return GIGA_OK;
  const uintptr_t es = dtype == GIGA_BF16 ? 2 : 4;
  struct P { const void* p; bool need; const char* name; uintptr_t align; };
  const P ps[] = {{im.x, (ops & (GIGA_OP_FWD | GIGA_OP_BWD_FILTER)) != 0, "x", es},
                  {im.y, (ops & GIGA_OP_FWD) != 0, "y", es},
                  {im.dy, (ops & (GIGA_OP_BWD_INPUT | GIGA_OP_BWD_FILTER)) != 0, "dy", es},
                  {im.dx, (ops & GIGA_OP_BWD_INPUT) != 0, "dx", es},
                  {im.w, (ops & (GIGA_OP_FWD | GIGA_OP_BWD_INPUT)) != 0, "w", 4},
                  {im.dw, (ops & GIGA_OP_BWD_FILTER) != 0, "dw", 4}};
  for (const P& p : ps) {
    if (!p.need) continue;
    if (!p.p) return fail(GIGA_ERR_INVALID_ARG, where + p.name + " is NULL");
    if (reinterpret_cast<uintptr_t>(p.p) % p.align)
      return fail(GIGA_ERR_MISALIGNED, where + p.name + " is misaligned");
  }
  const size_t bytes = (size_t)n * es;
  auto ov = [&](const void* a, const void* b) {
    if (!a || !b) return false;
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
  };
  if ((ops & GIGA_OP_FWD) && (ov(im.y, im.x) || ov(im.y, im.dy)))
    return fail(GIGA_ERR_INVALID_ARG, where + "y aliases an input");
  if ((ops & GIGA_OP_BWD_INPUT) && (ov(im.dx, im.dy) || ov(im.dx, im.x)))
    return fail(GIGA_ERR_INVALID_ARG, where + "dx aliases an input");
  return GIGA_OK;
}

int vec_image(const giga_image_t& im, int dtype) {
  if (im.W % 4) return 0;
  const uintptr_t align = dtype == GIGA_F32 ? 16 : 8;
  for (const void* p : {im.x, (const void*)im.y, im.dy, (const void*)im.dx})
    if (p && reinterpret_cast<uintptr_t>(p) % align) return 0;
  return 1;
}

// Builds everything but device state.  check_ptrs = false for size queries.
giga_status_t build_plan(const giga_image_t* images, int32_t n, int32_t ops, int32_t border,
                         int32_t dtype, bool check_ptrs, int tpc, giga_batched_plan_s* plan) {
  if (n < 0 || (n > 0 && !images)) return fail(GIGA_ERR_INVALID_ARG, "bad image list");
  if (ops <= 0 || (ops & ~(GIGA_OP_FWD | GIGA_OP_BWD_INPUT | GIGA_OP_BWD_FILTER)))
    return fail(GIGA_ERR_INVALID_ARG, "ops must be a non-empty GIGA_OP_* bitmask");
  if (border != GIGA_BORDER_ZERO && border != GIGA_BORDER_CLAMP)
    return fail(GIGA_ERR_INVALID_ARG, "unknown border");
  if (dtype != GIGA_F32 && dtype != GIGA_BF16) return fail(GIGA_ERR_INVALID_ARG, "unknown dtype");
  plan->ops = ops;
  plan->border = border;
  plan->dtype = dtype;
  plan->tpc = tpc;
  plan->images.resize(n);
  plan->chunks.clear();
  plan->empty_filter_grads.clear();
  plan->max_k = 1;
  std::vector<int64_t> tiles(n, 0);
  int64_t ic = 0, pf = 0, n_chunks = 0;
  for (int i = 0; i < n; ++i) {
    const giga_image_t& g = images[i];
    if (check_ptrs) {
      giga_status_t s = validate_image(g, i, ops, dtype);
      if (s != GIGA_OK) return s;
    } else if (g.K < 1 || g.K > kRagMaxK || g.K % 2 == 0 || g.H < 0 || g.W < 0 || g.C < 0) {
      return fail(GIGA_ERR_INVALID_ARG, "image " + std::to_string(i) + ": bad shape or K");
    }
    RagImage& r = plan->images[i];
    std::memset(&r, 0, sizeof(r));
    r.x = g.x; r.y = g.y; r.dy = g.dy; r.dx = g.dx; r.w = g.w; r.dw = g.dw;
    r.H = g.H; r.W = g.W; r.C = g.C; r.K = g.K;
    r.vec = vec_image(g, dtype);
    const int64_t px = (int64_t)g.H * g.W;
    if (px == 0 || g.C == 0) {
      if ((ops & GIGA_OP_BWD_FILTER) && g.C > 0) plan->empty_filter_grads.push_back(i);
      continue;
    }
    tiles[i] = ((g.W + kTileW - 1) / kTileW) * (int64_t)((g.H + kBwdTileH - 1) / kBwdTileH);
    r.nch = (int)((tiles[i] + tpc - 1) / tpc);
    r.ic_base = (int)ic;
    r.partial_base = pf;
    ic += g.C;
    if (ops & GIGA_OP_BWD_FILTER) pf += (int64_t)g.C * r.nch * g.K * g.K;
    n_chunks += (int64_t)g.C * r.nch;
    plan->max_k = std::max(plan->max_k, g.K);
  }
  if (n_chunks >= (1LL << 31) || ic >= (1LL << 30))
    return fail(GIGA_ERR_INVALID_ARG, "batch too large for one launch");
  // Longest first: chunks of the images with the largest per-pixel cost (K^2),
  // larger images first among equals; each image's chunks stay contiguous.
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int64_t ka = (int64_t)images[a].K * images[a].K, kb = (int64_t)images[b].K * images[b].K;
    if (ka != kb) return ka > kb;
    return tiles[a] > tiles[b];
  });
  plan->chunks.reserve((size_t)n_chunks);
  for (int i : order) {
    const RagImage& r = plan->images[i];
    if (tiles[i] == 0) continue;
    for (int c = 0; c < r.C; ++c)
      for (int j = 0; j < r.nch; ++j) {
        const int t0 = j * tpc;
        plan->chunks.push_back({i, c, t0, (int)std::min<int64_t>(t0 + tpc, tiles[i])});
      }
  }
  plan->n_ic = (int)ic;
  plan->partial_floats = pf;
  plan->off_chunks = align256(sizeof(RagImage) * (size_t)n);
  plan->off_counters = plan->off_chunks + align256(sizeof(RagChunk) * plan->chunks.size());
  plan->off_partials = plan->off_counters + align256(sizeof(int) * (size_t)(1 + ic));
  plan->ws_bytes = plan->off_partials + align256(sizeof(float) * (size_t)pf);
  plan->table_bytes = plan->off_counters;
  return GIGA_OK;
}

giga_status_t check_plan_ws(const giga_batched_plan_s* plan, void* ws, size_t ws_bytes) {
  if (!ws) return fail(GIGA_ERR_WORKSPACE, "workspace is NULL");
  if (ws_bytes < plan->ws_max)
    return fail(GIGA_ERR_WORKSPACE, "workspace too small, need " + std::to_string(plan->ws_max));
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return fail(GIGA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  return GIGA_OK;
}

// Tiles per chunk the plan can use; the autotuner times each of them.
constexpr int kRagTpcCandidates[] = {1, 2, 4, 8, 16, 32};

// Build the plan for tiles-per-chunk `tpc`, with workspace and table sizes
// that fit every candidate (the smallest chunks need the most of both).
giga_status_t build_plan_sized(const giga_image_t* images, int32_t n, int32_t ops,
                               int32_t border, int32_t dtype, bool check_ptrs, int tpc,
                               giga_batched_plan_s* plan) {
  giga_status_t s = build_plan(images, n, ops, border, dtype, check_ptrs, 1, plan);
  if (s != GIGA_OK) return s;
  const size_t ws_max = plan->ws_bytes, table_max = plan->table_bytes;
  if (tpc != 1 && (s = build_plan(images, n, ops, border, dtype, false, tpc, plan)) != GIGA_OK)
    return s;
  plan->ws_max = ws_max;
  plan->table_max = table_max;
  return GIGA_OK;
}

}  // namespace

extern "C" {

giga_status_t giga_batched_plan_create(const giga_image_t* images, int32_t n, int32_t ops,
                                       int32_t border, int32_t dtype,
                                       giga_batched_plan_t* plan) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  auto* p = new (std::nothrow) giga_batched_plan_s();
  if (!p) return fail(GIGA_ERR_INVALID_ARG, "out of host memory");
  giga_status_t s =
      build_plan_sized(images, n, ops, border, dtype, true, kRagTilesPerChunk, p);
  if (s != GIGA_OK) {
    delete p;
    return s;
  }
  if (n > 0) p->descs.assign(images, images + n);
  *plan = p;
  return GIGA_OK;
}

giga_status_t giga_batched_plan_workspace_size(giga_batched_plan_t plan, size_t* bytes) {
  clear_error();
  if (!plan || !bytes) return fail(GIGA_ERR_INVALID_ARG, "NULL argument");
  *bytes = plan->ws_max;
  return GIGA_OK;
}

giga_status_t giga_batched_plan_upload(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                       void* stream) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  giga_status_t s = check_plan_ws(plan, ws, ws_bytes);
  if (s != GIGA_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (plan->pending) {  // a previous upload may still read the pinned buffer
    if ((e = cudaEventSynchronize(plan->uploaded)) != cudaSuccess) return cuda_fail(e, "upload wait");
    plan->pending = false;
  }
  if (!plan->pinned) {
    if ((e = cudaMallocHost(&plan->pinned, plan->table_max)) != cudaSuccess)
      return cuda_fail(e, "pinned table");
    plan->pinned_bytes = plan->table_max;
  }
  // the table of the current chunk size (the autotuner rebuilds it)
  std::memset(plan->pinned, 0, plan->table_bytes);
  std::memcpy(plan->pinned, plan->images.data(), sizeof(RagImage) * plan->images.size());
  std::memcpy(static_cast<char*>(plan->pinned) + plan->off_chunks, plan->chunks.data(),
              sizeof(RagChunk) * plan->chunks.size());
  if (!plan->uploaded && (e = cudaEventCreateWithFlags(&plan->uploaded, cudaEventDisableTiming)))
    return cuda_fail(e, "event");
  if ((e = cudaMemcpyAsync(ws, plan->pinned, plan->table_bytes, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "table upload");
  if ((e = cudaEventRecord(plan->uploaded, st))) return cuda_fail(e, "event record");
  plan->pending = true;
  plan->uploaded_tpc = plan->tpc;
  plan->uploaded_ws = ws;
  return GIGA_OK;
}

giga_status_t giga_batched_plan_run(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                    void* stream) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  giga_status_t s = check_plan_ws(plan, ws, ws_bytes);
  if (s != GIGA_OK) return s;
  if (!plan->uploaded) return fail(GIGA_ERR_INVALID_ARG, "plan was never uploaded");
  // the kernels index the chunk table in the workspace: it must be this plan's
  if (plan->uploaded_tpc != plan->tpc)
    return fail(GIGA_ERR_INVALID_ARG, "the plan's table changed since its upload; upload it again");
  if (ws != plan->uploaded_ws)
    return fail(GIGA_ERR_WORKSPACE, "run with the workspace the table was uploaded to");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  cudaError_t e;
  for (int i : plan->empty_filter_grads) {
    const RagImage& r = plan->images[i];
    if ((e = cudaMemsetAsync(r.dw, 0, sizeof(float) * r.C * r.K * r.K, st)))
      return cuda_fail(e, "zeroing dw");
  }
  if (plan->chunks.empty()) return GIGA_OK;
  if ((e = cudaMemsetAsync(base + plan->off_counters, 0, sizeof(int) * (size_t)(1 + plan->n_ic), st)))
    return cuda_fail(e, "counter reset");
  RagParams p;
  p.images = reinterpret_cast<const RagImage*>(base);
  p.chunks = reinterpret_cast<const RagChunk*>(base + plan->off_chunks);
  p.counters = reinterpret_cast<int*>(base + plan->off_counters);
  p.partials = reinterpret_cast<float*>(base + plan->off_partials);
  p.n_chunks = (int)plan->chunks.size();
  p.tpc = plan->tpc;
  p.ops = plan->ops;
  p.border = plan->border;
  if (plan->max_k > kRagMaxK) return fail(GIGA_ERR_INVALID_ARG, "filter size above the batched limit");
  // one fixed layout, sized for the largest filter (two tile stages)
  const size_t smem = plan->dtype == GIGA_F32 ? rag_max_smem<float>()
                                               : rag_max_smem<__nv_bfloat16>();
  const int grid = (int)std::min<int64_t>((int64_t)sm_count(), (int64_t)plan->chunks.size());
  e = plan->dtype == GIGA_F32 ? rag_launch_f32(p, grid, smem, st)
                              : rag_launch_bf16(p, grid, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "ragged launch");
  return GIGA_OK;
}

void giga_batched_plan_destroy(giga_batched_plan_t plan) {
  if (!plan) return;
  if (plan->pending) cudaEventSynchronize(plan->uploaded);
  if (plan->uploaded) cudaEventDestroy(plan->uploaded);
  if (plan->pinned) cudaFreeHost(plan->pinned);
  delete plan;
}

giga_status_t giga_conv2d_batched(const giga_image_t* images, int32_t n, int32_t ops,
                                  int32_t border, int32_t dtype, void* ws, size_t ws_bytes,
                                  void* stream) {
  clear_error();
  giga_batched_plan_t plan = nullptr;
  giga_status_t s = giga_batched_plan_create(images, n, ops, border, dtype, &plan);
  if (s != GIGA_OK) return s;
  s = giga_batched_plan_upload(plan, ws, ws_bytes, stream);
  if (s == GIGA_OK) s = giga_batched_plan_run(plan, ws, ws_bytes, stream);
  std::string detail = giga_last_error_detail();
  giga_batched_plan_destroy(plan);
  if (s != GIGA_OK) fail(s, detail);
  return s;
}

giga_status_t giga_conv2d_batched_workspace_size(const giga_image_t* images, int32_t n,
                                                 int32_t ops, size_t* bytes) {
  clear_error();
  if (!bytes) return fail(GIGA_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  giga_batched_plan_s plan;
  giga_status_t s =
      build_plan_sized(images, n, ops, GIGA_BORDER_ZERO, GIGA_F32, false, kRagTilesPerChunk, &plan);
  if (s != GIGA_OK) return s;
  *bytes = plan.ws_max;
  return GIGA_OK;
}

giga_status_t giga_batched_plan_autotune(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                         void* stream, int32_t* tiles_per_chunk) {
  clear_error();
  if (!plan) return fail(GIGA_ERR_INVALID_ARG, "plan is NULL");
  giga_status_t s = check_plan_ws(plan, ws, ws_bytes);
  if (s != GIGA_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(e, "capture query");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(GIGA_ERR_INVALID_ARG, "the autotuner cannot run while the stream is capturing");
  const int n = (int)plan->descs.size();
  const giga_image_t* im = n ? plan->descs.data() : nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "event");
  float best_ms = 0.f;
  const int prev = plan->tpc;
  int best = prev;
  std::string times;
  for (int tpc : kRagTpcCandidates) {
    if ((s = build_plan(im, n, plan->ops, plan->border, plan->dtype, false, tpc, plan)) != GIGA_OK)
      break;
    if ((s = giga_batched_plan_upload(plan, ws, ws_bytes, stream)) != GIGA_OK) break;
    if ((s = giga_batched_plan_run(plan, ws, ws_bytes, stream)) != GIGA_OK) break;  // warm-up
    float ms = 0.f;
    cudaEventRecord(ev[0], st);
    for (int r = 0; r < 3 && s == GIGA_OK; ++r) s = giga_batched_plan_run(plan, ws, ws_bytes, stream);
    if (s != GIGA_OK) break;
    cudaEventRecord(ev[1], st);
    if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess) {
      s = cuda_fail(e, "autotune timing");
      break;
    }
    char buf[48];
    std::snprintf(buf, sizeof(buf), "%s%d:%.3f ms", times.empty() ? "" : " ", tpc, ms / 3.f);
    times += buf;
    if (tpc == kRagTpcCandidates[0] || ms < best_ms) {
      best_ms = ms;
      best = tpc;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (s != GIGA_OK) {
    // leave the plan describing its previous table; run() refuses it until the
    // caller uploads again, so no launch can read a table of another size
    const std::string detail = giga_last_error_detail();
    build_plan(im, n, plan->ops, plan->border, plan->dtype, false, prev, plan);
    plan->uploaded_tpc = 0;
    return fail(s, detail);
  }
  // rebuild and upload the chosen table
  if ((s = build_plan(im, n, plan->ops, plan->border, plan->dtype, false, best, plan)) != GIGA_OK)
    return s;
  if ((s = giga_batched_plan_upload(plan, ws, ws_bytes, stream)) != GIGA_OK) return s;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "autotune sync");
  if (tune_log_enabled())
    std::fprintf(stderr, "giga autotune: ragged batch of %d images -> %d tiles per chunk (%s)\n",
                 n, best, times.c_str());
  if (tiles_per_chunk) *tiles_per_chunk = best;
  return GIGA_OK;
}

int32_t giga_batched_plan_tiles_per_chunk(giga_batched_plan_t plan) {
  return plan ? plan->tpc : -1;
}

}  // extern "C"
