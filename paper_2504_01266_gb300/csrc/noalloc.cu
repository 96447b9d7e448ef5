// noalloc.cu -- filter gradient without a caller-provided workspace.
//
// giga_conv2d_bwd_filter needs a device workspace for its per-CTA partial
// sums, which the caller allocates.  Some callers cannot allocate device
// memory at the point where they need the gradient: code that runs under a
// fixed, pre-reserved memory budget (an inference/training server whose
// allocator owns all of HBM), plugins whose host framework exposes no
// workspace hook, and code on latency-critical paths where cudaMalloc's
// implicit device synchronisation is not acceptable.  This entry point serves
// them with a scratch buffer that lives in the library itself: a file-scope
// __device__ array of kNoAllocScratchBytes, created when the library's module
// is loaded on a device and held by that device until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "dw_launch.h"
#include "internal.h"

namespace giga {

// 4 MiB: room for 1M FP32 partial sums (e.g. 24 image planes x 128 CTAs x
// 225 taps of a 15 x 15 filter).
constexpr size_t kNoAllocScratchBytes = 4u << 20;
constexpr int64_t kNoAllocScratchFloats = (int64_t)(kNoAllocScratchBytes / sizeof(float));

static __device__ __align__(256) float g_filter_scratch[kNoAllocScratchFloats];

// Device address of g_filter_scratch, looked up once per device with that
// device current (the symbol's host-side name is not a device address).  The
// address is kept for the life of the process: after cudaDeviceReset the
// module is loaded again, possibly elsewhere, so the cached address no longer
// names the array (the header says so).
static std::mutex g_scratch_mu;
static void* g_scratch_ptr[64] = {};

static giga_status_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(GIGA_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GIGA_OK;
}

}  // namespace giga

using namespace giga;

extern "C" giga_status_t giga_conv2d_bwd_filter_noalloc(const giga_conv2d_desc_t* desc,
                                                        const void* x, const void* dy, float* dw,
                                                        void* stream) {
  clear_error();
  // The argument rules of giga_conv2d_bwd_filter, without its workspace.
  if (!desc) return fail(GIGA_ERR_INVALID_ARG, "desc is NULL");
  if (desc->reserved != 0) return fail(GIGA_ERR_INVALID_ARG, "desc.reserved must be 0");
  if (desc->N < 0 || desc->C_in < 0 || desc->H < 0 || desc->W < 0)
    return fail(GIGA_ERR_INVALID_ARG, "negative dimension");
  if (desc->H >= (1LL << 31) || desc->W >= (1LL << 31))
    return fail(GIGA_ERR_INVALID_ARG, "image too large");
  if (desc->K < 1 || desc->K > 31 || desc->K % 2 == 0)
    return fail(GIGA_ERR_INVALID_ARG, "K must be odd and in [1, 31]");
  if (desc->K > kMaxKFilter) return fail(GIGA_ERR_UNSUPPORTED, "the filter gradient supports K <= 15");
  if (desc->border != GIGA_BORDER_ZERO && desc->border != GIGA_BORDER_CLAMP)
    return fail(GIGA_ERR_INVALID_ARG, "unknown border");
  if (desc->dtype != GIGA_F32 && desc->dtype != GIGA_BF16)
    return fail(GIGA_ERR_INVALID_ARG, "unknown dtype");
  if (!(desc->groups == desc->C_in && desc->C_out == desc->C_in) ||
      desc->layout != GIGA_LAYOUT_NCHW)
    return fail(GIGA_ERR_UNSUPPORTED, "the allocation-free filter gradient is depthwise NCHW only");
  const int64_t planes = desc->N * desc->C_in;
  const int64_t kk = (int64_t)desc->K * desc->K;
  const int64_t n = planes * desc->H * desc->W;
  const size_t es = desc->dtype == GIGA_BF16 ? 2 : 4;
  if (desc->C_in > 0 && !dw) return fail(GIGA_ERR_INVALID_ARG, "dw is NULL");
  if (n > 0 && (!x || !dy)) return fail(GIGA_ERR_INVALID_ARG, "x or dy is NULL");
  if (reinterpret_cast<uintptr_t>(x) % es || reinterpret_cast<uintptr_t>(dy) % es ||
      reinterpret_cast<uintptr_t>(dw) % 4)
    return fail(GIGA_ERR_MISALIGNED, "x, dy or dw is not aligned to its element size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (desc->C_in == 0) return GIGA_OK;
    cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)(desc->C_in * kk), st);
    return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "zeroing dw");
  }

  DwArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = desc->N; a.C = desc->C_in; a.H = desc->H; a.W = desc->W; a.K = desc->K;
  a.border = desc->border; a.dtype = desc->dtype;
  // The chunking giga_conv2d_bwd_filter would use (the tuner's cached or
  // pinned choice; the built-in default if none, or with the tuner off; this
  // entry point never benchmarks), doubled until the partial sums fit the
  // scratch array.  A problem whose N*C*K*K partials alone exceed it is
  // refused.
  int id = tune_mode() == 0 ? 0 : tune_lookup(TUNE_BWD_FILTER, a);
  if (id < 0) id = 0;
  DwConfig cfg = tune_config(TUNE_BWD_FILTER, id, a);
  const int64_t tiles = dw_bwd_chunks_per_plane(desc->H, desc->W, 1);
  int64_t tpc = cfg.tiles_per_cta;
  while (planes * dw_bwd_chunks_per_plane(desc->H, desc->W, (int)tpc) * kk > kNoAllocScratchFloats &&
         tpc < tiles)
    tpc = std::min<int64_t>(tpc * 2, tiles);
  if (tpc >= (1LL << 31) ||
      planes * dw_bwd_chunks_per_plane(desc->H, desc->W, (int)tpc) * kk > kNoAllocScratchFloats)
    return fail(GIGA_ERR_INVALID_ARG,
                "problem too large for the allocation-free filter gradient: it needs more than "
                "the " + std::to_string(kNoAllocScratchFloats) + " partial sums of its scratch "
                "array (N*C*K*K = " + std::to_string(planes * kk) + "); use "
                "giga_conv2d_bwd_filter with a workspace");
  cfg.tiles_per_cta = (int)tpc;

  void* scratch = nullptr;
  giga_status_t s = scratch_address(&scratch);
  if (s != GIGA_OK) return s;
  a.x = x;
  a.dy = dy;
  a.dw = dw;
  // Every partial the finalize step reads is written by the same call first,
  // so the array needs no clearing between calls.
  a.partials = static_cast<float*>(scratch);
  const uintptr_t va = desc->dtype == GIGA_F32 ? 16 : 8;
  a.vec = (desc->W % 4 == 0 && reinterpret_cast<uintptr_t>(x) % va == 0 &&
           reinterpret_cast<uintptr_t>(dy) % va == 0) ? 1 : 0;
  return run_dw_op(TUNE_BWD_FILTER, a, cfg, st);
}
