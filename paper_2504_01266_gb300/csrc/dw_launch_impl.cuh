// dw_launch_impl.cuh -- launcher templates for the depthwise kernels; included
// only by the per-filter-size translation units dw_kNN.cu.
#pragma once

#include <algorithm>
#include <cstring>

#include "dw_kernels.cuh"
#include "dw_launch.h"

namespace giga {

// persistent = 0 (the default, fastest on the measured workloads): one tile
// per CTA and a single shared-memory stage (the kernel's prefetch branch never
// runs because gridDim.x >= tiles); 1: as many CTAs as fit on the GPU, each
// with two stages -- an autotuning candidate.
// The forward kernel of a launch: for FP32 K = 7 with one tile per CTA the
// five-CTA-per-SM compilation (instantiated for that case only), else the
// default one.  Raises the kernel's shared-memory limit first.
template <typename T, int K, int PY>
static cudaError_t fwd_kernel_for(bool persistent, size_t smem,
                                  decltype(&dw_fwd_kernel<T, K, PY>)* kern) {
  if constexpr (sizeof(T) == 4 && K == 7 && PY == 8) {
    if (!persistent) {
      *kern = dw_fwd_kernel_hi_occ<T, K, PY>;
      return set_smem_once<dw_fwd_kernel_hi_occ<T, K, PY>>(smem);
    }
  }
  *kern = dw_fwd_kernel<T, K, PY>;
  return set_smem_once<dw_fwd_kernel<T, K, PY>>(smem);
}

template <typename T, int K, int PY>
static cudaError_t fwd_impl(const DwArgs& a, bool input_grad, bool persistent, bool prefetch,
                            cudaStream_t st) {
  using S = FwdShape<K, PY, T>;
  decltype(&dw_fwd_kernel<T, K, PY>) kern = nullptr;
  cudaError_t e = fwd_kernel_for<T, K, PY>(persistent, (size_t)S::SM_BYTES, &kern);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + S::TH - 1) / S::TH;
  const int64_t tiles = a.N * a.C * tiles_x * tiles_y;
  int64_t grid = tiles;
  const size_t smem = persistent ? (size_t)S::SM_BYTES : (size_t)S::SM_BYTES_1;
  // resident CTAs per SM of this compilation at this shared-memory size
  // (per device, per persistence mode)
  static int ctas_per_sm[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63][persistent ? 1 : 0];
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kThreads, smem) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  const int64_t resident = (int64_t)per_sm * sm_count();
  if (persistent) grid = std::min<int64_t>(tiles, resident);
  // L2 prefetch distance in tiles (0: none): one tile per CTA -- the tile of
  // the CTA that starts when this one ends (one wave of resident CTAs
  // later); persistent -- this CTA's tile after next (the next is being
  // loaded).  A tuning option: it helps where the tile load's latency shows
  // (FP32 K = 7, 9) and costs where HBM is already saturated (K = 3).
  const int64_t pf = !prefetch ? 0 : persistent ? 2 * grid : resident;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const T* in = static_cast<const T*>(input_grad ? a.dy : a.x);
  T* out = static_cast<T*>(input_grad ? a.dx : a.y);
  // TMA staging for rows with a 16-byte stride from a 16-byte aligned base
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  int use_tma = 0;
  if (plane_tma_ok(in, sizeof(T), a.W))
    use_tma = make_plane_map(&tm, in, sizeof(T), a.W, a.H, a.N * a.C, Geo<K, sizeof(T)>::SP,
                             S::ROWS);
  kern<<<(unsigned)grid, kThreads, smem, st>>>(
      tm, in, a.w, out, make_fastdiv((uint32_t)a.C), (int)a.H, (int)a.W,
      make_fastdiv((uint32_t)tiles_x), make_fastdiv((uint32_t)tiles_y), tiles,
      input_grad ? 0 : a.border, a.vec, input_grad ? 1 : 0, use_tma, pf, dw_error_word());
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t dw_fwd_launch(const DwArgs& a, const DwConfig& cfg, bool input_grad,
                          cudaStream_t st) {
  const bool py4 = cfg.rows_per_thread == 4;
  const bool pers = cfg.persistent != 0, pf = cfg.prefetch != 0;
  if (a.dtype == 0)
    return py4 ? fwd_impl<float, K, 4>(a, input_grad, pers, pf, st)
               : fwd_impl<float, K, 8>(a, input_grad, pers, pf, st);
  return py4 ? fwd_impl<__nv_bfloat16, K, 4>(a, input_grad, pers, pf, st)
             : fwd_impl<__nv_bfloat16, K, 8>(a, input_grad, pers, pf, st);
}

template <typename T, int K>
static cudaError_t bwd_impl(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  using S = BwdShape<K, T>;
  const size_t smem = (size_t)S::SM_BYTES;
  auto kern = dw_bwd_kernel<T, K>;
  cudaError_t e = set_smem_once<dw_bwd_kernel<T, K>>(smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + kBwdTileH - 1) / kBwdTileH;
  const int64_t tpp = tiles_x * tiles_y;
  const int64_t chunks = dw_bwd_chunks_per_plane(a.H, a.W, cfg.tiles_per_cta);
  const int64_t grid = a.N * a.C * chunks;
  CUtensorMap tmx, tmdy;
  std::memset(&tmx, 0, sizeof(tmx));
  std::memset(&tmdy, 0, sizeof(tmdy));
  int use_tma = 0;
  constexpr int es = sizeof(T);
  if (plane_tma_ok(a.x, es, a.W) && plane_tma_ok(a.dy, es, a.W))
    use_tma = make_plane_map(&tmx, a.x, es, a.W, a.H, a.N * a.C, Geo<K, es>::SP, S::ROWS) &&
              make_plane_map(&tmdy, a.dy, es, a.W, a.H, a.N * a.C, Geo<K, es>::SP, S::ROWS);
  kern<<<(unsigned)grid, kThreads, smem, st>>>(
      tmx, tmdy, static_cast<const T*>(a.x), static_cast<const T*>(a.dy), a.w,
      static_cast<T*>(a.dx), a.partials, (int)a.C, (int)a.H, (int)a.W, (int)tiles_x, (int)tpp,
      (int)chunks, cfg.tiles_per_cta, a.border, a.vec, use_tma, dw_error_word());
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t dw_bwd_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  if constexpr (K > kMaxKFilter) {
    return cudaErrorInvalidValue;
  } else {
    return a.dtype == 0 ? bwd_impl<float, K>(a, cfg, st) : bwd_impl<__nv_bfloat16, K>(a, cfg, st);
  }
}

template <typename T, int K>
static cudaError_t bwd_ring_impl(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  using S = RingShape<K, T>;
  const size_t smem = (size_t)S::SM_BYTES;
  auto kern = dw_bwd_ring_kernel<T, K>;
  cudaError_t e = set_smem_once<dw_bwd_ring_kernel<T, K>>(smem);
  if (e != cudaSuccess) return e;
  static int ctas_per_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, S::NT, smem) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + kBwdTileH - 1) / kBwdTileH;
  const int64_t chunks = dw_bwd_chunks_per_plane(a.H, a.W, cfg.tiles_per_cta);
  const int64_t num_chunks = a.N * a.C * chunks;
  const int64_t grid = std::min<int64_t>(num_chunks, (int64_t)per_sm * sm_count());
  if (num_chunks + grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  CUtensorMap tmx, tmdy;
  std::memset(&tmx, 0, sizeof(tmx));
  std::memset(&tmdy, 0, sizeof(tmdy));
  int use_tma = 0;
  constexpr int es = sizeof(T);
  if (plane_tma_ok(a.x, es, a.W) && plane_tma_ok(a.dy, es, a.W))
    use_tma = make_plane_map(&tmx, a.x, es, a.W, a.H, a.N * a.C, Geo<K, es>::SP, S::ROWS) &&
              make_plane_map(&tmdy, a.dy, es, a.W, a.H, a.N * a.C, Geo<K, es>::SP, S::ROWS);
  kern<<<(unsigned)grid, S::NT, smem, st>>>(
      tmx, tmdy, static_cast<const T*>(a.x), static_cast<const T*>(a.dy), a.w,
      static_cast<T*>(a.dx), a.partials, (int)a.C, (int)a.H, (int)a.W,
      make_fastdiv((uint32_t)tiles_x), (int)(tiles_x * tiles_y), make_fastdiv((uint32_t)chunks),
      cfg.tiles_per_cta, (int)num_chunks, a.border, a.vec, use_tma, dw_error_word());
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t dw_bwd_ring_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  if constexpr (K > kMaxKFilter) {
    return cudaErrorInvalidValue;
  } else {
    return a.dtype == 0 ? bwd_ring_impl<float, K>(a, cfg, st)
                        : bwd_ring_impl<__nv_bfloat16, K>(a, cfg, st);
  }
}

template <typename T, int K>
static cudaError_t filter_impl(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  using S = FilterShape<K, T>;
  const size_t smem = (size_t)S::SM_BYTES;
  auto kern = dw_filter_kernel<T, K>;
  cudaError_t e = set_smem_once<dw_filter_kernel<T, K>>(smem);
  if (e != cudaSuccess) return e;
  static int ctas_per_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, S::NT, smem) !=
            cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + kFilterTileH - 1) / kFilterTileH;
  const int64_t chunks = dw_bwd_chunks_per_plane(a.H, a.W, cfg.tiles_per_cta);
  const int64_t num_chunks = a.N * a.C * chunks;
  const int64_t grid = std::min<int64_t>(num_chunks, (int64_t)per_sm * sm_count());
  if (num_chunks + grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  // TMA staging: rows with a 16-byte stride from 16-byte aligned bases;
  // otherwise cp.async staging.
  CUtensorMap tmx, tmdy;
  std::memset(&tmx, 0, sizeof(tmx));
  std::memset(&tmdy, 0, sizeof(tmdy));
  int use_tma = 0;
  constexpr int es = sizeof(T);
  if (plane_tma_ok(a.x, es, a.W) && plane_tma_ok(a.dy, es, a.W)) {
    use_tma = make_plane_map(&tmx, a.x, es, a.W, a.H, a.N * a.C, Geo<K, es>::SP, S::X_ROWS) &&
              make_plane_map(&tmdy, a.dy, es, a.W, a.H, a.N * a.C, kTileW, kFilterTileH);
  }
  int* err = dw_error_word();
  kern<<<(unsigned)grid, S::NT, smem, st>>>(
      tmx, tmdy, static_cast<const T*>(a.x), static_cast<const T*>(a.dy), a.partials, (int)a.H,
      (int)a.W, make_fastdiv((uint32_t)tiles_x), (int)(tiles_x * tiles_y),
      make_fastdiv((uint32_t)chunks), cfg.tiles_per_cta, (int)num_chunks, a.border, a.vec,
      use_tma, err);
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t dw_filter_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st) {
  if constexpr (K > kMaxKFilter) {
    return cudaErrorInvalidValue;
  } else {
    return a.dtype == 0 ? filter_impl<float, K>(a, cfg, st)
                        : filter_impl<__nv_bfloat16, K>(a, cfg, st);
  }
}

template <typename T, int K>
static cudaError_t sep_impl(const DwArgs& a, const float* wcol, const float* wrow,
                            cudaStream_t st) {
  using S = SepShape<K, T>;
  // FP32 K = 13, 15: the five-CTA compilation (instantiated for those only)
  decltype(&dw_sep_kernel<T, K>) kern = dw_sep_kernel<T, K>;
  cudaError_t e;
  if constexpr (sizeof(T) == 4 && (K == 13 || K == 15)) {
    kern = dw_sep_kernel_hi_occ<T, K>;
    e = set_smem_once<dw_sep_kernel_hi_occ<T, K>>((size_t)S::SM_BYTES);
  } else {
    e = set_smem_once<dw_sep_kernel<T, K>>((size_t)S::SM_BYTES);
  }
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + S::TH - 1) / S::TH;
  const int64_t grid = a.N * a.C * tiles_x * tiles_y;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  int use_tma = 0;
  if (plane_tma_ok(a.x, sizeof(T), a.W))
    use_tma = make_plane_map(&tm, a.x, sizeof(T), a.W, a.H, a.N * a.C, Geo<K, sizeof(T)>::SP,
                             S::ROWS);
  // L2 prefetch of the tile one wave of resident CTAs ahead: at K = 15 the
  // pass waits on its tile load (0.731 -> 0.700 ms on 8 x 3 x 4096^2); at
  // K = 3 and 7 it runs near the HBM rate and the prefetch costs 23 % / 15 %,
  // so only the largest filters use it
  static int ctas_per_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = ctas_per_sm[dev & 63];
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kThreads,
                                                      (size_t)S::SM_BYTES) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  const int pf = K >= 13 ? per_sm * sm_count() : 0;
  kern<<<(unsigned)grid, kThreads, (size_t)S::SM_BYTES, st>>>(
      tm, static_cast<const T*>(a.x), wcol, wrow, static_cast<T*>(a.y),
      make_fastdiv((uint32_t)a.C), (int)a.H, (int)a.W, make_fastdiv((uint32_t)tiles_x),
      make_fastdiv((uint32_t)tiles_y), a.border, a.vec, use_tma, pf, dw_error_word());
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t dw_sep_launch(const DwArgs& a, const float* wcol, const float* wrow,
                          cudaStream_t st) {
  return a.dtype == 0 ? sep_impl<float, K>(a, wcol, wrow, st)
                      : sep_impl<__nv_bfloat16, K>(a, wcol, wrow, st);
}

#define GIGA_DW_INSTANTIATE(K)                                                            \
  template cudaError_t dw_fwd_launch<K>(const DwArgs&, const DwConfig&, bool, cudaStream_t); \
  template cudaError_t dw_sep_launch<K>(const DwArgs&, const float*, const float*, cudaStream_t);
#define GIGA_DW_INSTANTIATE_BWD(K)                                                        \
  template cudaError_t dw_bwd_launch<K>(const DwArgs&, const DwConfig&, cudaStream_t);      \
  template cudaError_t dw_bwd_ring_launch<K>(const DwArgs&, const DwConfig&, cudaStream_t); \
  template cudaError_t dw_filter_launch<K>(const DwArgs&, const DwConfig&, cudaStream_t);

}  // namespace giga
