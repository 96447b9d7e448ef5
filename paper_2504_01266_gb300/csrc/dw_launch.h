// dw_launch.h -- host-side entry points of the depthwise kernels (one explicit
// instantiation per filter size lives in dw_kNN.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace giga {

constexpr int kMaxK = 31;        // forward / input gradient
constexpr int kMaxKFilter = 15;  // filter gradient and the batched path

// Forward (input_grad = false): y = K_w x with the border of `a`.
// Input gradient (input_grad = true): dx = g from dy (flipped filter, zero
// border); the clamp edge fold is a separate launch (dw_fixup_launch).
template <int K>
cudaError_t dw_fwd_launch(const DwArgs& a, const DwConfig& cfg, bool input_grad,
                          cudaStream_t st);

// Separable filter wcol (x) wrow [C][K] each: a row pass then a column pass
// in one launch (y = the forward with the outer-product filter, border of a).
template <int K>
cudaError_t dw_sep_launch(const DwArgs& a, const float* wcol, const float* wrow,
                          cudaStream_t st);

// Fused backward tile pass: g (the input gradient before the clamp edge
// fold) and the filter partials[planes * chunks][K*K].
template <int K>
cudaError_t dw_bwd_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st);

// Both gradients by the persistent kernel with a two-stage (x, dy) ring:
// g (the input gradient before the clamp edge fold) and the filter partials
// in the layout of dw_filter_launch (chunks of cfg.tiles_per_cta tiles).
template <int K>
cudaError_t dw_bwd_ring_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st);

// Filter gradient alone (persistent multi-stage kernel).  Writes
// partials[planes * chunks][K*K] in the same layout as dw_bwd_launch.
template <int K>
cudaError_t dw_filter_launch(const DwArgs& a, const DwConfig& cfg, cudaStream_t st);

// Upsampling by an integer factor s, alone or followed by the depthwise
// filter (upsample.cu).  N, C, H, W: the input; Ho = H * s, Wo = W * s.
struct UpArgs {
  const void* x;
  const float* w;
  void* y;
  int64_t N, C, H, W, Ho, Wo;
  int s, K, border, dtype, vec;
};
cudaError_t up_nearest_launch(const UpArgs& a, cudaStream_t st);
cudaError_t up_fwd_launch(const UpArgs& a, cudaStream_t st);

// RGB to grayscale, alone or followed by the filter (gray.cu): x is
// N x 3 x H x W, y is N x 1 x H x W, w is 1 x K x K.
struct GrayArgs {
  const void* x;
  const float* w;
  void* y;
  int64_t N, H, W;
  int K, border, dtype, vec;
};
cudaError_t gray_launch(const GrayArgs& a, cudaStream_t st);
cudaError_t gray_fwd_launch(const GrayArgs& a, cudaStream_t st);

// Device error word of the depthwise kernels (nonzero after a bounded wait
// gave up) for the current device; nullptr if unavailable.
int* dw_error_word();
// Synchronise `st`, read and clear that word.
cudaError_t dw_take_error(cudaStream_t st, int* code);
// Launch a kernel whose bounded mbarrier wait runs out (sets that word).
cudaError_t dw_wait_selftest(cudaStream_t st);

// Number of tile chunks per plane the backward pass uses for `tiles_per_cta`.
int64_t dw_bwd_chunks_per_plane(int64_t H, int64_t W, int tiles_per_cta);

// Clamp border: overwrite the edge pixels of dx with the exact adjoint.
cudaError_t dw_fixup_launch(const DwArgs& a, cudaStream_t st);

// dw[c][k] = sum over (n, chunk) of partials, in FP64, fixed order.
cudaError_t dw_finalize_launch(const DwArgs& a, int64_t chunks_per_plane, cudaStream_t st);

#define GIGA_DW_EXTERN(K)                                                                  \
  extern template cudaError_t dw_fwd_launch<K>(const DwArgs&, const DwConfig&, bool,      \
                                               cudaStream_t);                              \
  extern template cudaError_t dw_sep_launch<K>(const DwArgs&, const float*, const float*, \
                                               cudaStream_t);
#define GIGA_DW_EXTERN_BWD(K)                                                              \
  extern template cudaError_t dw_bwd_launch<K>(const DwArgs&, const DwConfig&,            \
                                               cudaStream_t);                              \
  extern template cudaError_t dw_bwd_ring_launch<K>(const DwArgs&, const DwConfig&,       \
                                                    cudaStream_t);                         \
  extern template cudaError_t dw_filter_launch<K>(const DwArgs&, const DwConfig&,         \
                                                  cudaStream_t);
GIGA_DW_EXTERN(1) GIGA_DW_EXTERN(3) GIGA_DW_EXTERN(5) GIGA_DW_EXTERN(7)
GIGA_DW_EXTERN(9) GIGA_DW_EXTERN(11) GIGA_DW_EXTERN(13) GIGA_DW_EXTERN(15)
GIGA_DW_EXTERN(17) GIGA_DW_EXTERN(19) GIGA_DW_EXTERN(21) GIGA_DW_EXTERN(23)
GIGA_DW_EXTERN(25) GIGA_DW_EXTERN(27) GIGA_DW_EXTERN(29) GIGA_DW_EXTERN(31)
GIGA_DW_EXTERN_BWD(1) GIGA_DW_EXTERN_BWD(3) GIGA_DW_EXTERN_BWD(5) GIGA_DW_EXTERN_BWD(7)
GIGA_DW_EXTERN_BWD(9) GIGA_DW_EXTERN_BWD(11) GIGA_DW_EXTERN_BWD(13) GIGA_DW_EXTERN_BWD(15)
#undef GIGA_DW_EXTERN
#undef GIGA_DW_EXTERN_BWD

}  // namespace giga
