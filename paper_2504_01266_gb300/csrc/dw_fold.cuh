// dw_fold.cuh -- clamp-border edge fold of the depthwise input gradient.
//
// With the clamp border the forward pass reads x at B(i + a - r), where B
// clamps a coordinate to [0, n).  Its adjoint returns w[a][b] * dy[i][j] to
// that clamped pixel, so the pixel p of an axis collects every (i, a) with
// B(i + a - r) = p:
//   p = 0     : i + a - r <= 0,   p = n - 1 : i + a - r >= n - 1,
//   otherwise : i + a - r == p    (both edge conditions when n == 1).
// For each filter row a those i form one interval, and the same holds for
// columns, so an edge pixel of dx is
//   dx[p][q] = sum_{a,b} w[a][b] * sum_{i in I(p,a)} sum_{j in J(q,b)} dy[i][j].
// The tile kernels compute the zero-border correlation everywhere; these
// helpers then overwrite the first/last row and column with the value above.
#pragma once

#include "common.cuh"

namespace giga {

__host__ __device__ __forceinline__ int64_t edge_pixels(int64_t H, int64_t W) {
  return (H == 1 || W == 1) ? H * W : 2 * W + 2 * (H - 2);
}

__device__ __forceinline__ void fold_interval(int p, int n, int a, int r, int& lo, int& hi) {
  const int ulo = (p == 0) ? -(1 << 30) : p;
  const int uhi = (p == n - 1) ? (1 << 30) : p;
  lo = max(0, ulo - a + r);
  hi = min(n - 1, uhi - a + r);
}

// Edge pixel number k of one plane: first row, last row, then the first and
// last column of the inner rows (alternating).
template <typename T>
__device__ __forceinline__ void fold_edge_pixel(const T* __restrict__ g,
                                                const float* __restrict__ f,
                                                T* __restrict__ d, int H, int W, int K,
                                                int64_t k) {
  const int r = (K - 1) / 2;
  int p, q;
  if (k < W) {
    p = 0;
    q = (int)k;
  } else if (H > 1 && k < 2 * (int64_t)W) {
    p = H - 1;
    q = (int)(k - W);
  } else {
    k -= (H > 1 ? 2 * (int64_t)W : W);
    p = 1 + (int)(k / (W > 1 ? 2 : 1));
    q = (W > 1 && (k & 1)) ? W - 1 : 0;
  }
  float sum = 0.f;
  for (int a = 0; a < K; ++a) {
    int ilo, ihi;
    fold_interval(p, H, a, r, ilo, ihi);
    if (ilo > ihi) continue;
    for (int b = 0; b < K; ++b) {
      int jlo, jhi;
      fold_interval(q, W, b, r, jlo, jhi);
      if (jlo > jhi) continue;
      float s = 0.f;
      for (int i = ilo; i <= ihi; ++i)
        for (int j = jlo; j <= jhi; ++j) s += Elem<T>::load(g + (int64_t)i * W + j);
      sum = fmaf(f[a * K + b], s, sum);
    }
  }
  Elem<T>::store(d + (int64_t)p * W + q, sum);
}

}  // namespace giga
