// api.cu -- the C ABI of libgiga (include/giga.h): argument validation,
// workspace sizing, dispatch to the depthwise kernels, status reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>

#include "dw_launch.h"
#include "internal.h"

namespace giga {

static thread_local std::string t_error;
static thread_local uint64_t t_launches = 0;

void note_launch(int n) { t_launches += (uint64_t)n; }

giga_status_t fail(giga_status_t status, const std::string& detail) {
  t_error = detail;
  return status;
}

giga_status_t cuda_fail(cudaError_t e, const char* where) {
  return fail(GIGA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void clear_error() { t_error.clear(); }

int sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int v = cached[dev].load();
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    cached[dev].store(v);
  }
  return v;
}

// ------------------------------------------------------------ validation

static bool is_depthwise(const giga_conv2d_desc_t* d) {
  return d->groups == d->C_in && d->C_out == d->C_in;
}

static giga_status_t check_desc(const giga_conv2d_desc_t* d) {
  if (!d) return fail(GIGA_ERR_INVALID_ARG, "desc is NULL");
  if (d->reserved != 0) return fail(GIGA_ERR_INVALID_ARG, "desc.reserved must be 0");
  if (d->N < 0 || d->C_in < 0 || d->C_out < 0 || d->H < 0 || d->W < 0)
    return fail(GIGA_ERR_INVALID_ARG, "negative dimension");
  if (d->K < 1 || d->K > 31 || (d->K % 2) == 0)
    return fail(GIGA_ERR_INVALID_ARG, "K must be odd and in [1, 31], got " + std::to_string(d->K));
  if (d->border != GIGA_BORDER_ZERO && d->border != GIGA_BORDER_CLAMP)
    return fail(GIGA_ERR_INVALID_ARG, "unknown border " + std::to_string(d->border));
  if (d->dtype != GIGA_F32 && d->dtype != GIGA_BF16)
    return fail(GIGA_ERR_INVALID_ARG, "unknown dtype " + std::to_string(d->dtype));
  if (d->layout != GIGA_LAYOUT_NCHW && d->layout != GIGA_LAYOUT_NHWC)
    return fail(GIGA_ERR_INVALID_ARG, "unknown layout " + std::to_string(d->layout));
  if (d->H >= (1LL << 31) || d->W >= (1LL << 31) || d->H * d->W >= (1LL << 40))
    return fail(GIGA_ERR_INVALID_ARG, "image too large");
  if (is_depthwise(d)) {
    if (d->layout != GIGA_LAYOUT_NCHW)
      return fail(GIGA_ERR_UNSUPPORTED, "depthwise filtering takes NCHW tensors");
    return GIGA_OK;
  }
  if (d->groups != 1)
    return fail(GIGA_ERR_INVALID_ARG, "groups must be C_in (depthwise, C_out == C_in) or 1 (dense)");
  return GIGA_OK;
}

static size_t elem_size(int dtype) { return dtype == GIGA_BF16 ? 2 : 4; }

static giga_status_t check_ptr(const void* p, size_t numel, size_t align, const char* name) {
  if (numel == 0) return GIGA_OK;
  if (!p) return fail(GIGA_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % align)
    return fail(GIGA_ERR_MISALIGNED, std::string(name) + " is not aligned to its element size");
  return GIGA_OK;
}

static bool overlap(const void* a, const void* b, size_t bytes) {
  if (!a || !b || bytes == 0) return false;
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

static int64_t dw_planes(const giga_conv2d_desc_t* d) { return d->N * d->C_in; }
static int64_t dw_numel(const giga_conv2d_desc_t* d) { return dw_planes(d) * d->H * d->W; }

static DwArgs make_args(const giga_conv2d_desc_t* d) {
  DwArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = d->N;
  a.C = d->C_in;
  a.H = d->H;
  a.W = d->W;
  a.K = d->K;
  a.border = d->border;
  a.dtype = d->dtype;
  return a;
}

// 128-bit (f32) / 64-bit (bf16) row accesses need aligned bases and W % 4 == 0.
static int vec_ok(const DwArgs& a, const void* p0, const void* p1, const void* p2) {
  const uintptr_t align = a.dtype == GIGA_F32 ? 16 : 8;
  if (a.W % 4) return 0;
  for (const void* p : {p0, p1, p2})
    if (p && reinterpret_cast<uintptr_t>(p) % align) return 0;
  return 1;
}

// Filter-gradient workspace: per-CTA partials at the smallest tiles-per-CTA
// any configuration uses (1), so every autotuner choice fits.
static size_t dw_filter_ws(const giga_conv2d_desc_t* d) {
  const int64_t chunks = dw_bwd_chunks_per_plane(d->H, d->W, 1);
  size_t bytes = (size_t)dw_planes(d) * (size_t)chunks * (size_t)(d->K * d->K) * sizeof(float);
  return (bytes + 255) / 256 * 256;
}

static giga_status_t check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return GIGA_OK;
  if (!ws) return fail(GIGA_ERR_WORKSPACE, "workspace is NULL, need " + std::to_string(need));
  if (ws_bytes < need)
    return fail(GIGA_ERR_WORKSPACE, "workspace of " + std::to_string(ws_bytes) +
                                        " bytes is too small, need " + std::to_string(need));
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return fail(GIGA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  return GIGA_OK;
}

// Dense path: 3 x 3, C_in = C_out = 64, BF16 NHWC, zero border; TMA needs
// 16-byte aligned tensors.
static giga_status_t check_dense(const giga_conv2d_desc_t* d) {
  if (d->C_in != 64 || d->C_out != 64 || d->K != 3)
    return fail(GIGA_ERR_UNSUPPORTED, "dense filtering supports 3 x 3 with C_in = C_out = 64");
  if (d->dtype != GIGA_BF16 || d->layout != GIGA_LAYOUT_NHWC)
    return fail(GIGA_ERR_UNSUPPORTED, "dense filtering takes BF16 NHWC tensors");
  if (d->border != GIGA_BORDER_ZERO)
    return fail(GIGA_ERR_UNSUPPORTED, "dense filtering supports the zero border");
  if (d->N >= (1LL << 31) || d->H >= (1LL << 31))
    return fail(GIGA_ERR_INVALID_ARG, "image too large");
  return GIGA_OK;
}

static giga_status_t check_dense_ptr(const void* p, size_t numel, const char* name) {
  if (numel == 0) return GIGA_OK;
  if (!p) return fail(GIGA_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 16)
    return fail(GIGA_ERR_MISALIGNED, std::string(name) + " must be 16-byte aligned (TMA)");
  return GIGA_OK;
}

static giga_status_t dense_run(const giga_conv2d_desc_t* d, const void* in, const void* w,
                               void* out, bool input_grad, void* ws, size_t ws_bytes,
                               void* stream) {
  giga_status_t s = check_dense(d);
  if (s != GIGA_OK) return s;
  const size_t n = (size_t)(d->N * d->H * d->W) * 64;
  if ((s = check_dense_ptr(in, n, input_grad ? "dy" : "x")) ||
      (s = check_dense_ptr(out, n, input_grad ? "dx" : "y")) ||
      (s = check_dense_ptr(w, n ? 64 * 9 * 64 : 0, "w")))
    return s;
  if (overlap(in, out, n * 2)) return fail(GIGA_ERR_INVALID_ARG, "output aliases the input");
  if (n == 0) return GIGA_OK;
  if (input_grad && (s = check_ws(ws, ws_bytes, dense_workspace_bytes(true)))) return s;
  cudaError_t e = dense_launch(in, w, out, d->N, d->H, d->W, input_grad, ws,
                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "dense launch");
  return GIGA_OK;
}

// --------------------------------------------------------------- dispatch

template <typename F>
static cudaError_t dispatch_k(int K, F&& f) {
  switch (K) {
#define GIGA_CASE(k) \
  case k:            \
    return f(std::integral_constant<int, k>{});
    GIGA_CASE(1) GIGA_CASE(3) GIGA_CASE(5) GIGA_CASE(7) GIGA_CASE(9) GIGA_CASE(11)
    GIGA_CASE(13) GIGA_CASE(15) GIGA_CASE(17) GIGA_CASE(19) GIGA_CASE(21) GIGA_CASE(23)
    GIGA_CASE(25) GIGA_CASE(27) GIGA_CASE(29) GIGA_CASE(31)
#undef GIGA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename F>
static cudaError_t dispatch_k_filter(int K, F&& f) {
  switch (K) {
#define GIGA_CASE(k) \
  case k:            \
    return f(std::integral_constant<int, k>{});
    GIGA_CASE(1) GIGA_CASE(3) GIGA_CASE(5) GIGA_CASE(7) GIGA_CASE(9) GIGA_CASE(11)
    GIGA_CASE(13) GIGA_CASE(15)
#undef GIGA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

giga_status_t run_dw_op(int op, const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  switch (op) {
    case TUNE_FWD:
      e = dispatch_k(a.K, [&](auto k) { return dw_fwd_launch<decltype(k)::value>(a, cfg, false, st); });
      if (e != cudaSuccess) return cuda_fail(e, "forward launch");
      return GIGA_OK;
    case TUNE_BWD_INPUT:
      e = dispatch_k(a.K, [&](auto k) { return dw_fwd_launch<decltype(k)::value>(a, cfg, true, st); });
      if (e == cudaSuccess) e = dw_fixup_launch(a, st);
      if (e != cudaSuccess) return cuda_fail(e, "input-gradient launch");
      return GIGA_OK;
    case TUNE_BWD_FILTER:
      e = dispatch_k_filter(a.K, [&](auto k) { return dw_filter_launch<decltype(k)::value>(a, cfg, st); });
      if (e == cudaSuccess)
        e = dw_finalize_launch(a, dw_bwd_chunks_per_plane(a.H, a.W, cfg.tiles_per_cta), st);
      if (e != cudaSuccess) return cuda_fail(e, "filter-gradient launch");
      return GIGA_OK;
    case TUNE_BWD_FUSED: {
      if (cfg.split) {
        // input gradient by the forward-style kernel, filter gradient by the
        // persistent filter kernel: two passes over dy, each role on its own
        // best kernel (faster for the ALU-bound large filters)
        // the input-gradient pass runs the forward kernel on a problem of the
        // same shape: take the forward's tuned configuration
        int fid = tune_mode() == 0 ? 0 : tune_lookup(TUNE_FWD, a);
        DwConfig fc = tune_config(TUNE_FWD, fid < 0 ? 0 : fid, a);
        giga_status_t s2 = run_dw_op(TUNE_BWD_INPUT, a, fc, st);
        if (s2 != GIGA_OK) return s2;
        return run_dw_op(TUNE_BWD_FILTER, a, cfg, st);
      }
      if (cfg.ring)
        e = dispatch_k_filter(a.K, [&](auto k) {
          return dw_bwd_ring_launch<decltype(k)::value>(a, cfg, st);
        });
      else
        e = dispatch_k_filter(a.K, [&](auto k) { return dw_bwd_launch<decltype(k)::value>(a, cfg, st); });
      if (e == cudaSuccess) e = dw_fixup_launch(a, st);
      if (e == cudaSuccess)
        e = dw_finalize_launch(a, dw_bwd_chunks_per_plane(a.H, a.W, cfg.tiles_per_cta), st);
      if (e != cudaSuccess) return cuda_fail(e, "backward launch");
      return GIGA_OK;
    }
  }
  return fail(GIGA_ERR_INVALID_ARG, "unknown op");
}

static bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus s = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &s) != cudaSuccess) return true;
  return s != cudaStreamCaptureStatusNone;
}

static giga_status_t run_tuned(int op, const DwArgs& a, cudaStream_t st) {
  int id = tune_mode() == 0 ? 0 : tune_lookup(op, a);
  if (id < 0 && tune_mode() == 2 && !stream_capturing(st)) {
    giga_status_t s = tune_dw_op(op, a, st);
    if (s != GIGA_OK) return s;
    id = tune_lookup(op, a);
  }
  if (id < 0) id = 0;
  return run_dw_op(op, a, tune_config(op, id, a), st);
}

}  // namespace giga

using namespace giga;

// ------------------------------------------------------------------ C ABI

extern "C" {

giga_status_t giga_conv2d_workspace_size(const giga_conv2d_desc_t* desc, int32_t ops,
                                         size_t* bytes) {
  clear_error();
  if (!bytes) return fail(GIGA_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (ops & ~(GIGA_OP_FWD | GIGA_OP_BWD_INPUT | GIGA_OP_BWD_FILTER))
    return fail(GIGA_ERR_INVALID_ARG, "unknown op bits");
  if (!is_depthwise(desc)) {
    if (ops & GIGA_OP_BWD_INPUT) *bytes = dense_workspace_bytes(true);
    if (ops & GIGA_OP_BWD_FILTER) *bytes = std::max(*bytes, dense_filter_workspace_bytes());
    return GIGA_OK;
  }
  if (ops & GIGA_OP_BWD_FILTER) *bytes = dw_filter_ws(desc);
  return GIGA_OK;
}

giga_status_t giga_conv2d_fwd(const giga_conv2d_desc_t* desc, const void* x, const void* w,
                              void* y, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc)) return dense_run(desc, x, w, y, false, ws, ws_bytes, stream);
  const size_t es = elem_size(desc->dtype);
  const size_t n = (size_t)dw_numel(desc);
  if ((s = check_ptr(x, n, es, "x")) || (s = check_ptr(y, n, es, "y")) ||
      (s = check_ptr(w, n ? (size_t)desc->C_in * desc->K * desc->K : 0, 4, "w")))
    return s;
  if (overlap(x, y, n * es)) return fail(GIGA_ERR_INVALID_ARG, "y aliases x");
  if (n == 0) return GIGA_OK;
  DwArgs a = make_args(desc);
  a.x = x;
  a.y = y;
  a.w = static_cast<const float*>(w);
  a.vec = vec_ok(a, x, y, nullptr);
  return run_tuned(TUNE_FWD, a, static_cast<cudaStream_t>(stream));
}

giga_status_t giga_conv2d_fwd_separable(const giga_conv2d_desc_t* desc, const void* x,
                                        const float* wcol, const float* wrow, void* y,
                                        void* stream) {
  clear_error();
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc))
    return fail(GIGA_ERR_UNSUPPORTED, "separable filters are depthwise (groups == C_in == C_out)");
  const size_t es = elem_size(desc->dtype);
  const size_t n = (size_t)dw_numel(desc);
  const size_t nw = n ? (size_t)desc->C_in * desc->K : 0;
  if ((s = check_ptr(x, n, es, "x")) || (s = check_ptr(y, n, es, "y")) ||
      (s = check_ptr(wcol, nw, 4, "wcol")) || (s = check_ptr(wrow, nw, 4, "wrow")))
    return s;
  if (overlap(x, y, n * es)) return fail(GIGA_ERR_INVALID_ARG, "y aliases x");
  if (n == 0) return GIGA_OK;
  DwArgs a = make_args(desc);
  a.x = x;
  a.y = y;
  a.vec = vec_ok(a, x, y, nullptr);
  cudaError_t e = dispatch_k(a.K, [&](auto k) {
    return dw_sep_launch<decltype(k)::value>(a, wcol, wrow, static_cast<cudaStream_t>(stream));
  });
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "separable launch");
}

// Shared checks of the two grayscale entry points; fills a.
static giga_status_t gray_prepare(const giga_conv2d_desc_t* desc, const void* x, const void* y,
                                  GrayArgs& a) {
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (desc->C_in != 3 || desc->C_out != 1 || desc->groups != 1)
    return fail(GIGA_ERR_INVALID_ARG, "grayscale takes C_in = 3 (R, G, B), C_out = 1, groups = 1");
  if (desc->layout != GIGA_LAYOUT_NCHW) return fail(GIGA_ERR_UNSUPPORTED, "grayscale takes NCHW");
  const size_t es = elem_size(desc->dtype);
  const size_t px = (size_t)(desc->N * desc->H * desc->W);
  if ((s = check_ptr(x, 3 * px, es, "x")) || (s = check_ptr(y, px, es, "y"))) return s;
  if (px && (reinterpret_cast<uintptr_t>(x) < reinterpret_cast<uintptr_t>(y) + px * es) &&
      (reinterpret_cast<uintptr_t>(y) < reinterpret_cast<uintptr_t>(x) + 3 * px * es))
    return fail(GIGA_ERR_INVALID_ARG, "y aliases x");
  std::memset(&a, 0, sizeof(a));
  a.x = x;
  a.y = const_cast<void*>(y);
  a.N = desc->N;
  a.H = desc->H;
  a.W = desc->W;
  a.K = desc->K;
  a.border = desc->border;
  a.dtype = desc->dtype;
  const uintptr_t align = desc->dtype == GIGA_F32 ? 16 : 8;
  a.vec = (desc->W % 4 == 0 && reinterpret_cast<uintptr_t>(x) % align == 0 &&
           reinterpret_cast<uintptr_t>(y) % align == 0) ? 1 : 0;
  return GIGA_OK;
}

giga_status_t giga_rgb_to_gray(const giga_conv2d_desc_t* desc, const void* x, void* y,
                               void* stream) {
  clear_error();
  GrayArgs a;
  giga_status_t s = gray_prepare(desc, x, y, a);
  if (s != GIGA_OK) return s;
  if (a.N * a.H * a.W == 0) return GIGA_OK;
  cudaError_t e = gray_launch(a, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "grayscale launch");
}

giga_status_t giga_gray_conv2d_fwd(const giga_conv2d_desc_t* desc, const void* x, const float* w,
                                   void* y, void* stream) {
  clear_error();
  GrayArgs a;
  giga_status_t s = gray_prepare(desc, x, y, a);
  if (s != GIGA_OK) return s;
  if (desc->K > kMaxKFilter)
    return fail(GIGA_ERR_UNSUPPORTED, "grayscale-then-filter supports K <= 15");
  const size_t px = (size_t)(a.N * a.H * a.W);
  if ((s = check_ptr(w, px ? (size_t)desc->K * desc->K : 0, 4, "w"))) return s;
  if (px == 0) return GIGA_OK;
  a.w = w;
  cudaError_t e = gray_fwd_launch(a, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "grayscale-then-filter launch");
}

// Shared checks of the two upsampling entry points; fills a.
static giga_status_t up_prepare(const giga_conv2d_desc_t* desc, int32_t scale, const void* x,
                                const void* y, UpArgs& a) {
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc))
    return fail(GIGA_ERR_UNSUPPORTED, "upsampling takes depthwise (per-channel) NCHW tensors");
  if (scale < 1) return fail(GIGA_ERR_INVALID_ARG, "scale must be >= 1, got " + std::to_string(scale));
  const int64_t Ho = desc->H * scale, Wo = desc->W * scale;
  if (Ho >= (1LL << 31) || Wo >= (1LL << 31) || Ho * Wo >= (1LL << 40))
    return fail(GIGA_ERR_INVALID_ARG, "upsampled image too large");
  const size_t es = elem_size(desc->dtype);
  const size_t n_in = (size_t)dw_numel(desc), n_out = (size_t)(dw_planes(desc) * Ho * Wo);
  if ((s = check_ptr(x, n_in, es, "x")) || (s = check_ptr(y, n_out, es, "y"))) return s;
  if (n_out && n_in && (reinterpret_cast<uintptr_t>(x) < reinterpret_cast<uintptr_t>(y) + n_out * es) &&
      (reinterpret_cast<uintptr_t>(y) < reinterpret_cast<uintptr_t>(x) + n_in * es))
    return fail(GIGA_ERR_INVALID_ARG, "y aliases x");
  std::memset(&a, 0, sizeof(a));
  a.x = x;
  a.y = const_cast<void*>(y);
  a.N = desc->N;
  a.C = desc->C_in;
  a.H = desc->H;
  a.W = desc->W;
  a.Ho = Ho;
  a.Wo = Wo;
  a.s = scale;
  a.K = desc->K;
  a.border = desc->border;
  a.dtype = desc->dtype;
  const uintptr_t align = desc->dtype == GIGA_F32 ? 16 : 8;
  a.vec = (Wo % 4 == 0 && reinterpret_cast<uintptr_t>(y) % align == 0) ? 1 : 0;
  return GIGA_OK;
}

giga_status_t giga_upsample_nearest(const giga_conv2d_desc_t* desc, int32_t scale, const void* x,
                                    void* y, void* stream) {
  clear_error();
  UpArgs a;
  giga_status_t s = up_prepare(desc, scale, x, y, a);
  if (s != GIGA_OK) return s;
  if (a.N * a.C * a.Ho * a.Wo == 0) return GIGA_OK;
  cudaError_t e = up_nearest_launch(a, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "upsample launch");
}

giga_status_t giga_upsample_conv2d_fwd(const giga_conv2d_desc_t* desc, int32_t scale,
                                       const void* x, const void* w, void* y, void* stream) {
  clear_error();
  UpArgs a;
  giga_status_t s = up_prepare(desc, scale, x, y, a);
  if (s != GIGA_OK) return s;
  if (desc->K > kMaxKFilter)
    return fail(GIGA_ERR_UNSUPPORTED, "upsample-then-filter supports K <= 15");
  const size_t n_out = (size_t)(a.N * a.C * a.Ho * a.Wo);
  if ((s = check_ptr(w, n_out ? (size_t)desc->C_in * desc->K * desc->K : 0, 4, "w"))) return s;
  if (n_out == 0) return GIGA_OK;
  if (scale == 1) {  // no upsampling: the plain depthwise forward, bit for bit
    DwArgs d = make_args(desc);
    d.x = x;
    d.y = y;
    d.w = static_cast<const float*>(w);
    d.vec = vec_ok(d, x, y, nullptr);
    return run_tuned(TUNE_FWD, d, static_cast<cudaStream_t>(stream));
  }
  a.w = static_cast<const float*>(w);
  cudaError_t e = up_fwd_launch(a, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "upsample-then-filter launch");
}

giga_status_t giga_conv2d_bwd_input(const giga_conv2d_desc_t* desc, const void* dy,
                                    const void* w, void* dx, void* ws, size_t ws_bytes,
                                    void* stream) {
  clear_error();
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc)) return dense_run(desc, dy, w, dx, true, ws, ws_bytes, stream);
  const size_t es = elem_size(desc->dtype);
  const size_t n = (size_t)dw_numel(desc);
  if ((s = check_ptr(dy, n, es, "dy")) || (s = check_ptr(dx, n, es, "dx")) ||
      (s = check_ptr(w, n ? (size_t)desc->C_in * desc->K * desc->K : 0, 4, "w")))
    return s;
  if (overlap(dy, dx, n * es)) return fail(GIGA_ERR_INVALID_ARG, "dx aliases dy");
  if (n == 0) return GIGA_OK;
  DwArgs a = make_args(desc);
  a.dy = dy;
  a.dx = dx;
  a.w = static_cast<const float*>(w);
  a.vec = vec_ok(a, dy, dx, nullptr);
  return run_tuned(TUNE_BWD_INPUT, a, static_cast<cudaStream_t>(stream));
}

static giga_status_t bwd_common(const giga_conv2d_desc_t* desc, const void* x, const void* dy,
                                const float* w, void* dx, float* dw, void* ws, size_t ws_bytes,
                                void* stream, bool fused) {
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc)) {
    if (fused) return fail(GIGA_ERR_UNSUPPORTED, "the fused backward pass is depthwise only");
    if ((s = check_dense(desc))) return s;
    const size_t n = (size_t)(desc->N * desc->H * desc->W) * 64;
    if ((s = check_dense_ptr(x, n, "x")) || (s = check_dense_ptr(dy, n, "dy")) ||
        (s = check_ptr(dw, 64 * 9 * 64, 4, "dw")))
      return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
      cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * 64 * 9 * 64, st);
      return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "zeroing dw");
    }
    if ((s = check_ws(ws, ws_bytes, dense_filter_workspace_bytes()))) return s;
    cudaError_t e = dense_wgrad_launch(x, dy, dw, desc->N, desc->H, desc->W, ws, st);
    return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "dense filter-gradient launch");
  }
  if (desc->K > kMaxKFilter)
    return fail(GIGA_ERR_UNSUPPORTED, "the filter gradient supports K <= 15");
  const size_t es = elem_size(desc->dtype);
  const size_t n = (size_t)dw_numel(desc);
  const size_t nw = (size_t)desc->C_in * desc->K * desc->K;
  if ((s = check_ptr(x, n, es, "x")) || (s = check_ptr(dy, n, es, "dy")) ||
      (s = check_ptr(dw, nw, 4, "dw")))
    return s;
  if (fused && ((s = check_ptr(dx, n, es, "dx")) || (s = check_ptr(w, n ? nw : 0, 4, "w"))))
    return s;
  if (fused && (overlap(dx, dy, n * es) || overlap(dx, x, n * es)))
    return fail(GIGA_ERR_INVALID_ARG, "dx aliases an input");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (nw) {
      cudaError_t e = cudaMemsetAsync(dw, 0, nw * sizeof(float), st);
      if (e != cudaSuccess) return cuda_fail(e, "zeroing dw");
    }
    return GIGA_OK;
  }
  if ((s = check_ws(ws, ws_bytes, dw_filter_ws(desc)))) return s;
  DwArgs a = make_args(desc);
  a.x = x;
  a.dy = dy;
  a.dx = dx;
  a.w = w;
  a.dw = dw;
  a.partials = static_cast<float*>(ws);
  a.vec = vec_ok(a, x, dy, fused ? dx : nullptr);
  return run_tuned(fused ? TUNE_BWD_FUSED : TUNE_BWD_FILTER, a, st);
}

giga_status_t giga_conv2d_bwd_filter(const giga_conv2d_desc_t* desc, const void* x,
                                     const void* dy, float* dw, void* ws, size_t ws_bytes,
                                     void* stream) {
  clear_error();
  return bwd_common(desc, x, dy, nullptr, nullptr, dw, ws, ws_bytes, stream, false);
}

giga_status_t giga_conv2d_bwd(const giga_conv2d_desc_t* desc, const void* x, const void* dy,
                              const float* w, void* dx, float* dw, void* ws, size_t ws_bytes,
                              void* stream) {
  clear_error();
  return bwd_common(desc, x, dy, w, dx, dw, ws, ws_bytes, stream, true);
}

static int tune_op_of(int32_t op) {
  switch (op) {
    case GIGA_OP_FWD: return TUNE_FWD;
    case GIGA_OP_BWD_INPUT: return TUNE_BWD_INPUT;
    case GIGA_OP_BWD_FILTER: return TUNE_BWD_FILTER;
    case GIGA_OP_BWD_INPUT | GIGA_OP_BWD_FILTER: return TUNE_BWD_FUSED;
    default: return -1;
  }
}

giga_status_t giga_autotune_conv2d(const giga_conv2d_desc_t* desc, int32_t ops, const void* x,
                                   const void* w, void* y, const void* dy, void* dx, float* dw,
                                   void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc)) return fail(GIGA_ERR_UNSUPPORTED, "only depthwise problems are tuned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (stream_capturing(st)) return fail(GIGA_ERR_UNSUPPORTED, "cannot autotune while capturing");
  if (dw_numel(desc) == 0) return GIGA_OK;
  // Validate every requested op exactly like its entry point (one run each).
  if ((ops & GIGA_OP_FWD) && (s = giga_conv2d_fwd(desc, x, w, y, ws, ws_bytes, stream))) return s;
  const bool fused = (ops & GIGA_OP_BWD_INPUT) && (ops & GIGA_OP_BWD_FILTER);
  if (fused) {
    if ((s = giga_conv2d_bwd(desc, x, dy, static_cast<const float*>(w), dx, dw, ws, ws_bytes, stream)))
      return s;
  } else {
    if ((ops & GIGA_OP_BWD_INPUT) && (s = giga_conv2d_bwd_input(desc, dy, w, dx, ws, ws_bytes, stream)))
      return s;
    if ((ops & GIGA_OP_BWD_FILTER) &&
        (s = giga_conv2d_bwd_filter(desc, x, dy, dw, ws, ws_bytes, stream)))
      return s;
  }
  DwArgs a = make_args(desc);
  a.x = x; a.y = y; a.dy = dy; a.dx = dx; a.w = static_cast<const float*>(w); a.dw = dw;
  a.partials = static_cast<float*>(ws);
  a.vec = vec_ok(a, x, y, nullptr) && vec_ok(a, dy, dx, nullptr);
  if ((ops & GIGA_OP_FWD) && (s = tune_dw_op(TUNE_FWD, a, st))) return s;
  if (fused) return tune_dw_op(TUNE_BWD_FUSED, a, st);
  if ((ops & GIGA_OP_BWD_INPUT) && (s = tune_dw_op(TUNE_BWD_INPUT, a, st))) return s;
  if ((ops & GIGA_OP_BWD_FILTER) && (s = tune_dw_op(TUNE_BWD_FILTER, a, st))) return s;
  return GIGA_OK;
}

int32_t giga_autotune_choice(const giga_conv2d_desc_t* desc, int32_t op) {
  clear_error();
  if (check_desc(desc) != GIGA_OK || !is_depthwise(desc)) return -1;
  const int top = tune_op_of(op);
  if (top < 0) return -1;
  if (tune_mode() == 0) return 0;
  const int id = tune_lookup(top, make_args(desc));
  return id < 0 ? 0 : id;
}

giga_status_t giga_autotune_set_choice(const giga_conv2d_desc_t* desc, int32_t op, int32_t id) {
  clear_error();
  giga_status_t s = check_desc(desc);
  if (s != GIGA_OK) return s;
  if (!is_depthwise(desc)) return fail(GIGA_ERR_UNSUPPORTED, "only depthwise problems are tuned");
  const int top = tune_op_of(op);
  if (top < 0) return fail(GIGA_ERR_INVALID_ARG, "op must be 1, 2, 4 or 6");
  if (id < 0 || id >= tune_candidates(top))
    return fail(GIGA_ERR_INVALID_ARG, "configuration id " + std::to_string(id) + " out of range");
  tune_store(top, make_args(desc), id);
  return GIGA_OK;
}

const char* giga_status_string(giga_status_t status) {
  switch (status) {
    case GIGA_OK: return "success";
    case GIGA_ERR_INVALID_ARG: return "invalid argument";
    case GIGA_ERR_UNSUPPORTED: return "unsupported configuration";
    case GIGA_ERR_MISALIGNED: return "misaligned pointer";
    case GIGA_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case GIGA_ERR_CUDA: return "CUDA error";
    case GIGA_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* giga_last_error_detail(void) { return t_error.c_str(); }

giga_status_t giga_check_device_error(void* stream) {
  clear_error();
  int code = 0, dw_code = 0;
  cudaError_t e = dense_take_error(static_cast<cudaStream_t>(stream), &code);
  if (e == cudaSuccess) e = dw_take_error(static_cast<cudaStream_t>(stream), &dw_code);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  if (code != 0)
    return fail(GIGA_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on a pipeline barrier");
  if (dw_code != 0)
    return fail(GIGA_ERR_TIMEOUT, "a depthwise kernel gave up waiting for a TMA tile copy");
  return GIGA_OK;
}

giga_status_t giga_selftest_bounded_wait(void* stream) {
  clear_error();
  cudaError_t e = dw_wait_selftest(static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GIGA_OK : cuda_fail(e, "bounded-wait self-test launch");
}

uint64_t giga_launch_count(void) { return t_launches; }

void giga_launch_count_reset(void) { t_launches = 0; }

}  // extern "C"
