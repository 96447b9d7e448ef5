// dw_misc.cu -- the two small kernels around the depthwise backward pass:
//  * the clamp-border edge fold of the input gradient, and
//  * the FP64 fixed-order reduction of the per-CTA filter-gradient partials.
#include <algorithm>

#include "dw_fold.cuh"
#include "dw_kernels.cuh"
#include "dw_launch.h"
#include "tma.cuh"

namespace giga {

// Device error word of the depthwise kernels (bounded TMA waits).
static __device__ int g_dw_err;

int* dw_error_word() {
  static int* cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cached[dev]) {
    int* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_dw_err) != cudaSuccess) return nullptr;
    cached[dev] = p;
  }
  return cached[dev];
}

cudaError_t dw_take_error(cudaStream_t st, int* code) {
  *code = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  int* err = dw_error_word();
  if (!err) return cudaErrorInvalidSymbol;
  e = cudaMemcpy(code, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpy(err, &zero, sizeof(int), cudaMemcpyHostToDevice);
}

// One thread waits on an mbarrier that nothing ever completes: the bounded
// wait gives up after kWaitLimitNs and records kDevErrTimeout, exercising the
// same path a stalled TMA load would take.
__global__ void dw_wait_selftest_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  if (!mbar_wait(&bar, 0)) record_error(err, kDevErrTimeout);
}

cudaError_t dw_wait_selftest(cudaStream_t st) {
  int* err = dw_error_word();
  if (!err) return cudaErrorInvalidSymbol;
  dw_wait_selftest_kernel<<<1, 32, 0, st>>>(err);
  note_launch();
  return cudaGetLastError();
}

int64_t dw_bwd_chunks_per_plane(int64_t H, int64_t W, int tiles_per_cta) {
  const int64_t tiles = ((W + kTileW - 1) / kTileW) * ((H + kBwdTileH - 1) / kBwdTileH);
  return (tiles + tiles_per_cta - 1) / tiles_per_cta;
}

// ------------------------------------------------------------- edge fold
template <typename T>
__global__ void dw_fixup_kernel(const T* __restrict__ dy, const float* __restrict__ w,
                                T* __restrict__ dx, int C, int H, int W, int K,
                                int64_t edge_per_plane, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t plane = e / edge_per_plane;
    const int64_t k = e - plane * edge_per_plane;
    fold_edge_pixel<T>(dy + plane * (int64_t)H * W, w + (int64_t)(plane % C) * K * K,
                       dx + plane * (int64_t)H * W, H, W, K, k);
  }
}

// ---- FP32 clamp fold as corrections on top of the zero-border values g that
// the tile pass already wrote.  With g[u][v] = sum_{a,b} w[a][b] dy[u-a+r][v-b+r]
// (dy zero outside) on the extended domain, the clamp adjoint is
// dx[p][q] = sum_{u: B(u)=p} sum_{v: B(v)=q} g[u][v], i.e. g plus the margin sums
//   top     T[q] = sum_{i<r}  sum_b Wt[i][b] dy[i][q-b+r],     Wt[i][b] = sum_{a<=r-1-i} w[a][b]
//   bottom  B[q] = sum_{d<r}  sum_b Wb[d][b] dy[H-1-d][q-b+r], Wb[d][b] = sum_{a>=r+1+d} w[a][b]
//   left    L[p] = sum_{j<r}  sum_a Wl[j][a] dy[p-a+r][j],     Wl[j][a] = sum_{b<=r-1-j} w[a][b]
//   right   R[p] = sum_{e<r}  sum_a Wr[e][a] dy[p-a+r][W-1-e], Wr[e][a] = sum_{b>=r+1+e} w[a][b]
// and at the corners the doubly-folded sums, e.g.
//   TL = sum_{i<r,j<r} (sum_{a<=r-1-i} sum_{b<=r-1-j} w[a][b]) dy[i][j]
// (i, d < H and j, e < W; dy outside the image reads zero).  The row kernel adds
// T and B to the first and last row; the column kernel, launched after it,
// adds L, R and the corner sums to the first and last column.
constexpr int kFoldThreads = 256;

__device__ __forceinline__ float dy_at(const float* g, int H, int W, int i, int j) {
  return (i >= 0 && i < H && j >= 0 && j < W) ? g[(int64_t)i * W + j] : 0.f;
}

__global__ void dw_fold_rows_kernel(const float* __restrict__ dy, const float* __restrict__ w,
                                    float* __restrict__ dx, int C, int H, int W, int K) {
  extern __shared__ float tab[];  // Wt[r][K], Wb[r][K]
  const int r = (K - 1) / 2;
  const int64_t plane = blockIdx.y;
  const float* f = w + (plane % C) * (int64_t)K * K;
  float* Wt = tab;
  float* Wb = tab + r * K;
  for (int k = threadIdx.x; k < r * K; k += blockDim.x) {
    const int i = k / K, b = k % K;
    float t = 0.f, u = 0.f;
    for (int a = 0; a <= r - 1 - i; ++a) t += f[a * K + b];
    for (int a = r + 1 + i; a < K; ++a) u += f[a * K + b];
    Wt[k] = t;
    Wb[k] = u;
  }
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W) return;
  const float* g = dy + plane * (int64_t)H * W;
  const int rows = min(r, H);
  float top = 0.f, bot = 0.f;
  for (int i = 0; i < rows; ++i)
    for (int b = 0; b < K; ++b) {
      top = fmaf(Wt[i * K + b], dy_at(g, H, W, i, q - b + r), top);
      bot = fmaf(Wb[i * K + b], dy_at(g, H, W, H - 1 - i, q - b + r), bot);
    }
  float* d = dx + plane * (int64_t)H * W;
  if (H == 1) {
    d[q] += top + bot;
  } else {
    d[q] += top;
    d[(int64_t)(H - 1) * W + q] += bot;
  }
}

__global__ void dw_fold_cols_kernel(const float* __restrict__ dy, const float* __restrict__ w,
                                    float* __restrict__ dx, int C, int H, int W, int K) {
  extern __shared__ float tab[];  // Wl[r][K], Wr[r][K], corners 4 x r x r, two row strips
  const int r = (K - 1) / 2;
  const int64_t plane = blockIdx.y;
  const float* f = w + (plane % C) * (int64_t)K * K;
  float* Wl = tab;
  float* Wr = tab + r * K;
  float* Ctl = tab + 2 * r * K;
  float* Ctr = Ctl + r * r;
  float* Cbl = Ctr + r * r;
  float* Cbr = Cbl + r * r;
  for (int k = threadIdx.x; k < r * K; k += blockDim.x) {
    const int j = k / K, a = k % K;
    float l = 0.f, rr = 0.f;
    for (int b = 0; b <= r - 1 - j; ++b) l += f[a * K + b];
    for (int b = r + 1 + j; b < K; ++b) rr += f[a * K + b];
    Wl[k] = l;
    Wr[k] = rr;
  }
  for (int k = threadIdx.x; k < r * r; k += blockDim.x) {
    const int i = k / r, j = k % r;
    float tl = 0.f, tr = 0.f, bl = 0.f, br = 0.f;
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) {
        const float v = f[a * K + b];
        const bool top = a <= r - 1 - i, bottom = a >= r + 1 + i;
        const bool left = b <= r - 1 - j, right = b >= r + 1 + j;
        if (top && left) tl += v;
        if (top && right) tr += v;
        if (bottom && left) bl += v;
        if (bottom && right) br += v;
      }
    Ctl[k] = tl;
    Ctr[k] = tr;
    Cbl[k] = bl;
    Cbr[k] = br;
  }
  // the block's rows p0 - r .. p0 + blockDim.x - 1 + r of the first and the
  // last r columns, staged once (neighbouring threads share K - 1 of their K
  // rows; reading them from global memory per thread was latency-bound)
  const float* g = dy + plane * (int64_t)H * W;
  const int cols = min(r, W), rows = min(r, H);
  const int p0 = blockIdx.x * blockDim.x;
  const int strip_rows = blockDim.x + 2 * r;
  float* sl = Cbr + r * r;           // [strip_rows][r]: columns 0 .. r - 1
  float* sr = sl + strip_rows * r;   // [strip_rows][r]: columns W - 1 .. W - r
  for (int k = threadIdx.x; k < strip_rows * r; k += blockDim.x) {
    const int i = k / r, j = k - (k / r) * r;
    const int row = p0 - r + i;
    sl[k] = j < cols ? dy_at(g, H, W, row, j) : 0.f;
    sr[k] = j < cols ? dy_at(g, H, W, row, W - 1 - j) : 0.f;
  }
  __syncthreads();
  const int p = p0 + threadIdx.x;
  if (p >= H) return;
  float left = 0.f, right = 0.f;
  for (int j = 0; j < cols; ++j)
    for (int a = 0; a < K; ++a) {
      // dy row p - a + r sits at strip row threadIdx.x + 2r - a
      const int i = threadIdx.x + 2 * r - a;
      left = fmaf(Wl[j * K + a], sl[i * r + j], left);
      right = fmaf(Wr[j * K + a], sr[i * r + j], right);
    }
  // corner sums belong to the pixels of the first / last row
  if (p == 0 || p == H - 1) {
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < cols; ++j) {
        if (p == 0) {
          left = fmaf(Ctl[i * r + j], dy_at(g, H, W, i, j), left);
          right = fmaf(Ctr[i * r + j], dy_at(g, H, W, i, W - 1 - j), right);
        }
        if (p == H - 1) {
          left = fmaf(Cbl[i * r + j], dy_at(g, H, W, H - 1 - i, j), left);
          right = fmaf(Cbr[i * r + j], dy_at(g, H, W, H - 1 - i, W - 1 - j), right);
        }
      }
  }
  float* d = dx + plane * (int64_t)H * W + (int64_t)p * W;
  if (W == 1) {
    d[0] += left + right;
  } else {
    d[0] += left;
    d[W - 1] += right;
  }
}

cudaError_t dw_fixup_launch(const DwArgs& a, cudaStream_t st) {
  if (a.border != 1 || a.N * a.C * a.H * a.W == 0) return cudaSuccess;
  const int r = (a.K - 1) / 2;
  if (a.dtype == 0 && r > 0 && a.N * a.C <= 65535) {
    const int64_t planes = a.N * a.C;
    const dim3 grid_rows((unsigned)((a.W + kFoldThreads - 1) / kFoldThreads), (unsigned)planes);
    const dim3 grid_cols((unsigned)((a.H + kFoldThreads - 1) / kFoldThreads), (unsigned)planes);
    dw_fold_rows_kernel<<<grid_rows, kFoldThreads, sizeof(float) * 2 * r * a.K, st>>>(
        static_cast<const float*>(a.dy), a.w, static_cast<float*>(a.dx), (int)a.C, (int)a.H,
        (int)a.W, a.K);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t cols_smem =
        sizeof(float) * (2 * r * a.K + 4 * r * r + 2 * (kFoldThreads + 2 * r) * r);
    dw_fold_cols_kernel<<<grid_cols, kFoldThreads, cols_smem, st>>>(
        static_cast<const float*>(a.dy), a.w, static_cast<float*>(a.dx), (int)a.C, (int)a.H,
        (int)a.W, a.K);
    note_launch();
    return cudaGetLastError();
  }
  const int64_t H = a.H, W = a.W;
  const int64_t edge = edge_pixels(H, W);
  const int64_t total = a.N * a.C * edge;
  const int threads = 128;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 65535);
  if (a.dtype == 0)
    dw_fixup_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const float*>(a.dy), a.w, static_cast<float*>(a.dx), (int)a.C, (int)H,
        (int)W, a.K, edge, total);
  else
    dw_fixup_kernel<__nv_bfloat16><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const __nv_bfloat16*>(a.dy), a.w, static_cast<__nv_bfloat16*>(a.dx),
        (int)a.C, (int)H, (int)W, a.K, edge, total);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------ FP64 reduction
// One warp per (channel, tap): lanes stride over the (image, chunk) partials
// in a fixed order, accumulate in FP64 and combine with a fixed butterfly, so
// the result does not depend on scheduling.
__global__ void dw_finalize_kernel(const float* __restrict__ partials, float* __restrict__ dw,
                                   int64_t N, int C, int64_t chunks, int KK) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)C * KK) return;
  const int c = (int)(gw / KK), k = (int)(gw % KK);
  double s = 0.0;
  const int64_t count = N * chunks;
  // idx = n * chunks + ch advances by 32 = step_n * chunks + step_ch: one
  // division per lane instead of a 64-bit division per partial
  int64_t n = lane / chunks, ch = lane - (lane / chunks) * chunks;
  const int64_t step_n = 32 / chunks, step_ch = 32 - step_n * chunks;
  for (int64_t idx = lane; idx < count; idx += 32) {
    s += (double)partials[((n * C + c) * chunks + ch) * KK + k];
    n += step_n;
    ch += step_ch;
    if (ch >= chunks) {
      ch -= chunks;
      ++n;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) dw[(int64_t)c * KK + k] = (float)s;
}

cudaError_t dw_finalize_launch(const DwArgs& a, int64_t chunks_per_plane, cudaStream_t st) {
  const int KK = a.K * a.K;
  const int64_t warps = a.C * KK;
  const int threads = 256;
  const int64_t blocks = (warps * 32 + threads - 1) / threads;
  dw_finalize_kernel<<<(unsigned)blocks, threads, 0, st>>>(a.partials, a.dw, a.N, (int)a.C,
                                                           chunks_per_plane, KK);
  note_launch();
  return cudaGetLastError();
}

}  // namespace giga
