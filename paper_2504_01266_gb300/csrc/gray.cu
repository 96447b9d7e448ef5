// gray.cu -- RGB to grayscale (the GigaAPI paper, Section 4.2.5) alone and
// fused in front of the depthwise filter: the filter runs on the gray image,
// whose pixels are formed while a tile is staged, so the gray image never
// goes to HBM.
//
//   gray[n][i][j] = 0.299 x[n][0][i][j] + 0.587 x[n][1][i][j] + 0.114 x[n][2][i][j]
//   y[n][0][i][j] = sum_{a,b} w[a][b] * gray~[n][i + a - r][j + b - r]
//
// gray~ applies the border rule on the gray image (zero, or clamp; both
// commute with the per-pixel weighted sum).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "dw_kernels.cuh"
#include "dw_launch.h"

namespace giga {

constexpr float kGrayR = 0.299f, kGrayG = 0.587f, kGrayB = 0.114f;

__device__ __forceinline__ float gray_of(float r, float g, float b) {
  return fmaf(kGrayB, b, fmaf(kGrayG, g, kGrayR * r));
}

// ------------------------------------------------------------ conversion
// Image n = blockIdx.y, + gridDim.y, ...; pixels grid-strided along x (no
// division per pixel).
template <typename T>
__global__ void __launch_bounds__(256) gray_kernel(const T* __restrict__ x, T* __restrict__ y,
                                                   int64_t P, int64_t N) {
  for (int64_t n = blockIdx.y; n < N; n += gridDim.y) {
    const T* xn = x + n * 3 * P;
    T* yn = y + n * P;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x)
      Elem<T>::store(yn + p, gray_of(Elem<T>::load(xn + p), Elem<T>::load(xn + P + p),
                                     Elem<T>::load(xn + 2 * P + p)));
  }
}

// ------------------------------------------------ grayscale, then filter
// One 32 x 128 tile of the gray image per CTA (8 warps, 4 rows each).  The
// three channel tiles (with the halo) are staged as three consecutive
// slices -- one TMA load with a box three planes deep, or cp.async -- then
// every staged cell becomes its gray value (FP32: in place over the red
// slice; BF16: into a separate FP32 tile in the compute geometry).
template <int K, typename T>
struct GrayShape {
  using G = Geo<K>;
  using GS = Geo<K, sizeof(T)>;
  static constexpr int PY = 4;
  static constexpr int TH = kWarps * PY;
  static constexpr int ROWS = TH + 2 * G::R;
  static constexpr int SLICE = ROWS * GS::SP * (int)sizeof(T);  // one staged channel
  static constexpr int HEAD = 128;                               // mbarrier, abort flag
  static constexpr int STAGED = HEAD;
  static constexpr int GRAY = sizeof(T) == 4 ? STAGED : round_up(STAGED + 3 * SLICE, 128);
  static constexpr int W_OFF =
      round_up(std::max(STAGED + 3 * SLICE, GRAY + ROWS * G::SP * 4), 16);
  static constexpr int SM_BYTES = W_OFF + G::WPAD * 4;
};

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) gray_fwd_kernel(
    const __grid_constant__ CUtensorMap tmx, const T* __restrict__ x, const float* __restrict__ w,
    T* __restrict__ y, int H, int W, FastDiv ftx, FastDiv fty, int clamp, int vec, int use_tma,
    int* err) {
  using G = Geo<K>;
  using GS = Geo<K, sizeof(T)>;
  using S = GrayShape<K, T>;
  extern __shared__ __align__(128) float smem[];
  char* sm = reinterpret_cast<char*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + 8);
  T* staged = reinterpret_cast<T*>(sm + S::STAGED);
  float* gt = reinterpret_cast<float*>(sm + S::GRAY);
  float* sw = reinterpret_cast<float*>(sm + S::W_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x;
  const uint32_t t2 = fdiv(t, ftx);
  const int tx0 = (int)(t - t2 * ftx.d) * kTileW;
  const uint32_t nu = fdiv(t2, fty);
  const int ty0 = (int)(t2 - nu * fty.d) * S::TH;
  const int64_t n = nu;

  stage_filter_async<K>(sw, w, false, kThreads);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  cta_barrier();
  if (use_tma) {
    cp_async_commit();
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, (uint32_t)(3 * S::SLICE));
      tma_load_3d(staged, &tmx, tx0 - GS::RP, ty0 - G::R, (int)(3 * n), bar);
    }
    cp_async_wait_all();
    if (!mbar_wait(bar, 0)) {
      record_error(err, kDevErrTimeout);
      *s_abort = 1;
    }
  } else {
    constexpr int SLICE_ELEMS = S::ROWS * GS::SP;
#pragma unroll 1
    for (int ch = 0; ch < 3; ++ch)
      stage_tile<T, G::R, GS::RP, GS::SP, kThreads, false>(
          staged + ch * SLICE_ELEMS, x + (3 * n + ch) * (int64_t)H * W, H, W, ty0, tx0, S::ROWS,
          clamp != 0, vec != 0);
    cp_async_commit();
    cp_async_wait_all();
  }
  cta_barrier();
  if (*s_abort) {
    mbar_wait(bar, 0);  // let a late copy land (bounded) before the CTA exits
    return;
  }
  // gray value of every staged cell, in 4-element chunks (column c of the
  // FP32 tile is staged column c + D)
  {
    constexpr int SLICE_ELEMS = S::ROWS * GS::SP;
    constexpr int D = GS::RP - G::RP;
    constexpr int CPR = G::SP / 4;
    for (int k = threadIdx.x; k < S::ROWS * CPR; k += kThreads) {
      const int r = k / CPR, c = (k - (k / CPR) * CPR) * 4;
      const T* p0 = staged + r * GS::SP + c + D;
      const float4 a = Tile<T>::load4(p0);
      const float4 b = Tile<T>::load4(p0 + SLICE_ELEMS);
      const float4 d = Tile<T>::load4(p0 + 2 * SLICE_ELEMS);
      *reinterpret_cast<float4*>(gt + r * G::SP + c) =
          make_float4(gray_of(a.x, b.x, d.x), gray_of(a.y, b.y, d.y), gray_of(a.z, b.z, d.z),
                      gray_of(a.w, b.w, d.w));
    }
  }
  cta_barrier();
  if (use_tma && clamp &&
      (ty0 - G::R < 0 || ty0 + S::TH + G::R > H || tx0 - G::RP < 0 || tx0 + kTileW + G::RP > W))
    clamp_fix<float, G::SP, kThreads>(gt, H, W, ty0, tx0, G::R, G::RP, S::ROWS);
  float acc[S::PY][4];
  fwd_block<K, S::PY, float>(gt + warp * S::PY * G::SP + 4 * lane, sw, acc);
  store_block<T, S::PY>(y + n * (int64_t)H * W, H, W, ty0 + warp * S::PY, tx0 + 4 * lane,
                        vec != 0, acc);
}

template <typename T, int K>
static cudaError_t gray_fwd_impl(const GrayArgs& a, cudaStream_t st) {
  using S = GrayShape<K, T>;
  cudaError_t e = set_smem_once<gray_fwd_kernel<T, K>>((size_t)S::SM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.W + kTileW - 1) / kTileW;
  const int64_t tiles_y = (a.H + S::TH - 1) / S::TH;
  const int64_t grid = a.N * tiles_x * tiles_y;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  int use_tma = 0;
  if (plane_tma_ok(a.x, sizeof(T), a.W)) {
    // the box is three planes deep: the R, G and B tiles of one image in one load
    EncodeFn enc = encode_fn();
    if (enc) {
      const int es = (int)sizeof(T);
      cuuint64_t dims[3] = {(cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)(3 * a.N)};
      cuuint64_t strides[2] = {(cuuint64_t)(a.W * es), (cuuint64_t)(a.H * a.W * es)};
      cuuint32_t box[3] = {(cuuint32_t)Geo<K, sizeof(T)>::SP, (cuuint32_t)S::ROWS, 3};
      cuuint32_t estr[3] = {1, 1, 1};
      use_tma = enc(&tm, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    3, const_cast<void*>(a.x), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
  }
  gray_fwd_kernel<T, K><<<(unsigned)grid, kThreads, (size_t)S::SM_BYTES, st>>>(
      tm, static_cast<const T*>(a.x), a.w, static_cast<T*>(a.y), (int)a.H, (int)a.W,
      make_fastdiv((uint32_t)tiles_x), make_fastdiv((uint32_t)tiles_y), a.border, a.vec, use_tma,
      dw_error_word());
  note_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t gray_fwd_dispatch(const GrayArgs& a, cudaStream_t st) {
  switch (a.K) {
    case 1: return gray_fwd_impl<T, 1>(a, st);
    case 3: return gray_fwd_impl<T, 3>(a, st);
    case 5: return gray_fwd_impl<T, 5>(a, st);
    case 7: return gray_fwd_impl<T, 7>(a, st);
    case 9: return gray_fwd_impl<T, 9>(a, st);
    case 11: return gray_fwd_impl<T, 11>(a, st);
    case 13: return gray_fwd_impl<T, 13>(a, st);
    case 15: return gray_fwd_impl<T, 15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gray_fwd_launch(const GrayArgs& a, cudaStream_t st) {
  return a.dtype == 0 ? gray_fwd_dispatch<float>(a, st)
                      : gray_fwd_dispatch<__nv_bfloat16>(a, st);
}

cudaError_t gray_launch(const GrayArgs& a, cudaStream_t st) {
  const int64_t P = a.H * a.W;
  // about 16 CTAs of 256 threads per SM in all, split between images (y) and
  // the pixels of an image (x)
  const int64_t budget = (int64_t)sm_count() * 16;
  const int64_t gy = std::min<int64_t>(a.N, 65535);
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, budget / gy + 1));
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (a.dtype == 0)
    gray_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(a.x),
                                             static_cast<float*>(a.y), P, a.N);
  else
    gray_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
        static_cast<const __nv_bfloat16*>(a.x), static_cast<__nv_bfloat16*>(a.y), P, a.N);
  note_launch();
  return cudaGetLastError();
}

}  // namespace giga
