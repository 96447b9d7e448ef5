/*
 * giga_oracle.c -- FP64 reference implementation of dense 2D image filtering.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA library under paper_2504_01266_gb300/csrc, and it never calls it.
 *
 * What it computes (GigaAPI paper, Section 4.2.4 "Sharpening"): every output
 * pixel of every colour channel is the weighted sum of the pixels of a square
 * neighbourhood centred on it, each neighbour multiplied by the filter entry at
 * the same relative position; neighbours that fall outside the image are
 * skipped.  Skipping an out-of-image neighbour is the same as reading a zero
 * there (the "zero" border).  The widened operation adds:
 *   - a K x K filter for any odd K (the paper uses 3 x 3), one filter per
 *     channel (depthwise), shared by every image of the batch;
 *   - a "clamp" border: an out-of-image neighbour reads the nearest edge pixel
 *     (row and column clamped independently);
 *   - the two adjoints needed for training: the gradient with respect to the
 *     input (the transpose of the forward operator) and the gradient with
 *     respect to the filter;
 *   - the dense multi-channel case (every output channel sums over every input
 *     channel), which is the same neighbourhood sum with one more index;
 *   - nearest-neighbour upsampling by an integer factor (Section 4.2.3), and
 *     the paper's sharpening benchmark (Section 6.6): the filter applied to
 *     the upsampled image;
 *   - RGB to grayscale conversion (Section 4.2.5), the luminance weights
 *     0.299, 0.587, 0.114 of the red, green and blue channels.
 *
 * Conventions (plain definitions, no blocking or reordering):
 *   r = (K - 1) / 2, tap (a, b) with a, b in [0, K) reads the neighbour at
 *   (i + a - r, j + b - r): a cross-correlation, the filter is not flipped.
 *   Depthwise tensors are NCHW, the filter is w[c][a][b].
 *   Dense tensors are NHWC, the filter is w[o][a][b][c].
 *
 * Everything is double precision.  OpenMP splits work only across whole
 * outputs (or across planes whose outputs no other thread touches), so every
 * output is summed in the same order as the serial loop.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_ZERO 0
#define ORACLE_CLAMP 1

/* Where does the neighbour at coordinate p (possibly outside [0, n)) read
 * from?  Returns 1 and sets *src when it reads a pixel, 0 when the zero
 * border skips it.  Clamp maps every outside coordinate to the nearest edge. */
static int border_source(int64_t p, int64_t n, int border, int64_t* src) {
    if (p >= 0 && p < n) { *src = p; return 1; }
    if (border == ORACLE_ZERO) return 0;
    *src = p < 0 ? 0 : n - 1;
    return 1;
}

static int check_args(int64_t N, int64_t C, int64_t H, int64_t W, int K, int border) {
    if (N < 0 || C < 0 || H < 0 || W < 0) return 1;
    if (K < 1 || (K % 2) == 0) return 1;
    if (border != ORACLE_ZERO && border != ORACLE_CLAMP) return 1;
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- depthwise */

/* One forward output: y[n][c][i][j] = sum_{a,b} w[c][a][b] * x~[n][c][i+a-r][j+b-r]. */
static double dw_fwd_one(const double* x, const double* w, int64_t C, int64_t H, int64_t W,
                         int K, int border, int64_t n, int64_t c, int64_t i, int64_t j) {
    const int r = (K - 1) / 2;
    const double* plane = x + (n * C + c) * H * W;
    const double* f = w + c * (int64_t)K * K;
    double sum = 0.0;
    for (int a = 0; a < K; ++a) {
        int64_t si;
        if (!border_source(i + a - r, H, border, &si)) continue;
        for (int b = 0; b < K; ++b) {
            int64_t sj;
            if (!border_source(j + b - r, W, border, &sj)) continue;
            sum += f[a * K + b] * plane[si * W + sj];
        }
    }
    return sum;
}

int oracle_dw_fwd(const double* x, const double* w, double* y, int64_t N, int64_t C,
                  int64_t H, int64_t W, int K, int border) {
    if (check_args(N, C, H, W, K, border)) return 1;
    int64_t rows = N * C * H;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t i = row % H, nc = row / H, c = nc % C, n = nc / C;
        for (int64_t j = 0; j < W; ++j)
            y[row * W + j] = dw_fwd_one(x, w, C, H, W, K, border, n, c, i, j);
    }
    return 0;
}

/* Forward outputs at selected flat NCHW indices only (for spot checks of
 * workloads too large to evaluate in full). */
int oracle_dw_fwd_points(const double* x, const double* w, int64_t N, int64_t C, int64_t H,
                         int64_t W, int K, int border, const int64_t* idx, int64_t count,
                         double* out) {
    if (check_args(N, C, H, W, K, border)) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        int64_t f = idx[t];
        int64_t j = f % W, i = (f / W) % H, c = (f / (W * H)) % C, n = f / (W * H * C);
        out[t] = dw_fwd_one(x, w, C, H, W, K, border, n, c, i, j);
    }
    return 0;
}

/* Gradient with respect to the input, as the transpose of the forward map.
 * The forward pass sends w[c][a][b] * x~[src] to y[i][j]; the transpose sends
 * w[c][a][b] * dy[i][j] back to the pixel src it was read from.  Written as
 * this scatter on purpose: the zero border drops the contribution, the clamp
 * border piles it onto the edge pixel it was read from.  Planes are
 * independent, so threads split over (n, c) only. */
int oracle_dw_bwd_input(const double* dy, const double* w, double* dx, int64_t N, int64_t C,
                        int64_t H, int64_t W, int K, int border) {
    if (check_args(N, C, H, W, K, border)) return 1;
    const int r = (K - 1) / 2;
    int64_t planes = N * C;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < planes; ++p) {
        const int64_t c = p % C;
        const double* g = dy + p * H * W;
        double* d = dx + p * H * W;
        const double* f = w + c * (int64_t)K * K;
        for (int64_t q = 0; q < H * W; ++q) d[q] = 0.0;
        for (int64_t i = 0; i < H; ++i)
            for (int64_t j = 0; j < W; ++j)
                for (int a = 0; a < K; ++a) {
                    int64_t si;
                    if (!border_source(i + a - r, H, border, &si)) continue;
                    for (int b = 0; b < K; ++b) {
                        int64_t sj;
                        if (!border_source(j + b - r, W, border, &sj)) continue;
                        d[si * W + sj] += f[a * K + b] * g[i * W + j];
                    }
                }
    }
    return 0;
}

/* The same transpose evaluated at single pixels: collect, for the pixel
 * (p, q), exactly the scatter contributions above whose source is (p, q).
 * Any (i, a) with source p has |i - p| <= r, so the search stays local. */
int oracle_dw_bwd_input_points(const double* dy, const double* w, int64_t N, int64_t C,
                               int64_t H, int64_t W, int K, int border, const int64_t* idx,
                               int64_t count, double* out) {
    if (check_args(N, C, H, W, K, border)) return 1;
    const int r = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        int64_t f = idx[t];
        int64_t q = f % W, p = (f / W) % H, c = (f / (W * H)) % C, n = f / (W * H * C);
        const double* g = dy + (n * C + c) * H * W;
        const double* fw = w + c * (int64_t)K * K;
        double sum = 0.0;
        for (int64_t i = p - r; i <= p + r; ++i) {
            if (i < 0 || i >= H) continue;
            for (int64_t j = q - r; j <= q + r; ++j) {
                if (j < 0 || j >= W) continue;
                for (int a = 0; a < K; ++a) {
                    int64_t si;
                    if (!border_source(i + a - r, H, border, &si) || si != p) continue;
                    for (int b = 0; b < K; ++b) {
                        int64_t sj;
                        if (!border_source(j + b - r, W, border, &sj) || sj != q) continue;
                        sum += fw[a * K + b] * g[i * W + j];
                    }
                }
            }
        }
        out[t] = sum;
    }
    return 0;
}

/* One filter-gradient tap: dw[c][a][b] = sum_{n,i,j} dy[n][c][i][j] * x~[n][c][i+a-r][j+b-r].
 * The filter is shared by the whole batch, so the sum runs over n as well. */
static double dw_filter_one(const double* x, const double* dy, int64_t N, int64_t C,
                            int64_t H, int64_t W, int K, int border, int64_t c, int a, int b) {
    const int r = (K - 1) / 2;
    double sum = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        const double* xp = x + (n * C + c) * H * W;
        const double* gp = dy + (n * C + c) * H * W;
        for (int64_t i = 0; i < H; ++i) {
            int64_t si;
            if (!border_source(i + a - r, H, border, &si)) continue;
            for (int64_t j = 0; j < W; ++j) {
                int64_t sj;
                if (!border_source(j + b - r, W, border, &sj)) continue;
                sum += gp[i * W + j] * xp[si * W + sj];
            }
        }
    }
    return sum;
}

int oracle_dw_bwd_filter(const double* x, const double* dy, double* dw, int64_t N, int64_t C,
                         int64_t H, int64_t W, int K, int border) {
    if (check_args(N, C, H, W, K, border)) return 1;
    int64_t taps = C * (int64_t)K * K;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < taps; ++t) {
        int64_t c = t / ((int64_t)K * K);
        int a = (int)((t / K) % K), b = (int)(t % K);
        dw[t] = dw_filter_one(x, dy, N, C, H, W, K, border, c, a, b);
    }
    return 0;
}

/* Selected taps only (flat index c*K*K + a*K + b). */
int oracle_dw_bwd_filter_taps(const double* x, const double* dy, int64_t N, int64_t C, int64_t H,
                              int64_t W, int K, int border, const int64_t* tap, int64_t count,
                              double* out) {
    if (check_args(N, C, H, W, K, border)) return 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < count; ++t) {
        int64_t c = tap[t] / ((int64_t)K * K);
        int a = (int)((tap[t] / K) % K), b = (int)(tap[t] % K);
        out[t] = dw_filter_one(x, dy, N, C, H, W, K, border, c, a, b);
    }
    return 0;
}

/* -------------------------------------------------------------------- dense */

/* y[n][i][j][o] = sum_{a,b,c} w[o][a][b][c] * x~[n][i+a-r][j+b-r][c]  (NHWC). */
static double dense_fwd_one(const double* x, const double* w, int64_t H, int64_t W, int64_t Ci,
                            int K, int border, int64_t n, int64_t i, int64_t j, int64_t o) {
    const int r = (K - 1) / 2;
    double sum = 0.0;
    for (int a = 0; a < K; ++a) {
        int64_t si;
        if (!border_source(i + a - r, H, border, &si)) continue;
        for (int b = 0; b < K; ++b) {
            int64_t sj;
            if (!border_source(j + b - r, W, border, &sj)) continue;
            const double* px = x + ((n * H + si) * W + sj) * Ci;
            const double* f = w + ((o * K + a) * (int64_t)K + b) * Ci;
            for (int64_t c = 0; c < Ci; ++c) sum += f[c] * px[c];
        }
    }
    return sum;
}

int oracle_dense_fwd(const double* x, const double* w, double* y, int64_t N, int64_t H,
                     int64_t W, int64_t Ci, int64_t Co, int K, int border) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
    int64_t pix = N * H * W;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < pix; ++p) {
        int64_t j = p % W, i = (p / W) % H, n = p / (W * H);
        for (int64_t o = 0; o < Co; ++o)
            y[p * Co + o] = dense_fwd_one(x, w, H, W, Ci, K, border, n, i, j, o);
    }
    return 0;
}

int oracle_dense_fwd_points(const double* x, const double* w, int64_t N, int64_t H, int64_t W,
                            int64_t Ci, int64_t Co, int K, int border, const int64_t* idx,
                            int64_t count, double* out) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        int64_t f = idx[t];
        int64_t o = f % Co, p = f / Co;
        int64_t j = p % W, i = (p / W) % H, n = p / (W * H);
        out[t] = dense_fwd_one(x, w, H, W, Ci, K, border, n, i, j, o);
    }
    return 0;
}

/* Transpose of the dense forward map, as a scatter (see oracle_dw_bwd_input). */
int oracle_dense_bwd_input(const double* dy, const double* w, double* dx, int64_t N, int64_t H,
                           int64_t W, int64_t Ci, int64_t Co, int K, int border) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
    const int r = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double* d = dx + n * H * W * Ci;
        for (int64_t q = 0; q < H * W * Ci; ++q) d[q] = 0.0;
        for (int64_t i = 0; i < H; ++i)
            for (int64_t j = 0; j < W; ++j) {
                const double* g = dy + ((n * H + i) * W + j) * Co;
                for (int a = 0; a < K; ++a) {
                    int64_t si;
                    if (!border_source(i + a - r, H, border, &si)) continue;
                    for (int b = 0; b < K; ++b) {
                        int64_t sj;
                        if (!border_source(j + b - r, W, border, &sj)) continue;
                        double* px = d + (si * W + sj) * Ci;
                        for (int64_t o = 0; o < Co; ++o) {
                            const double* f = w + ((o * K + a) * (int64_t)K + b) * Ci;
                            for (int64_t c = 0; c < Ci; ++c) px[c] += f[c] * g[o];
                        }
                    }
                }
            }
    }
    return 0;
}

/* One dense filter-gradient tap (flat index ((o*K + a)*K + b)*Ci + c):
 * dw[o][a][b][c] = sum_{n,i,j} dy[n][i][j][o] * x~[n][i+a-r][j+b-r][c]. */
static double dense_filter_one(const double* x, const double* dy, int64_t N, int64_t H,
                               int64_t W, int64_t Ci, int64_t Co, int K, int border, int64_t t) {
    const int r = (K - 1) / 2;
    int64_t c = t % Ci, b = (t / Ci) % K, a = (t / (Ci * K)) % K, o = t / (Ci * K * K);
    double sum = 0.0;
    for (int64_t n = 0; n < N; ++n)
        for (int64_t i = 0; i < H; ++i) {
            int64_t si;
            if (!border_source(i + a - r, H, border, &si)) continue;
            for (int64_t j = 0; j < W; ++j) {
                int64_t sj;
                if (!border_source(j + b - r, W, border, &sj)) continue;
                sum += dy[((n * H + i) * W + j) * Co + o] * x[((n * H + si) * W + sj) * Ci + c];
            }
        }
    return sum;
}

int oracle_dense_bwd_filter(const double* x, const double* dy, double* dw, int64_t N, int64_t H,
                            int64_t W, int64_t Ci, int64_t Co, int K, int border) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
    int64_t taps = Co * (int64_t)K * K * Ci;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < taps; ++t)
        dw[t] = dense_filter_one(x, dy, N, H, W, Ci, Co, K, border, t);
    return 0;
}

int oracle_dense_bwd_filter_taps(const double* x, const double* dy, int64_t N, int64_t H,
                                 int64_t W, int64_t Ci, int64_t Co, int K, int border,
                                 const int64_t* tap, int64_t count, double* out) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < count; ++t)
        out[t] = dense_filter_one(x, dy, N, H, W, Ci, Co, K, border, tap[t]);
    return 0;
}

/* The dense transpose at single NHWC elements (p, q, c): the scatter
 * contributions of oracle_dense_bwd_input whose source pixel is (p, q). */
int oracle_dense_bwd_input_points(const double* dy, const double* w, int64_t N, int64_t H,
                                  int64_t W, int64_t Ci, int64_t Co, int K, int border,
                                  const int64_t* idx, int64_t count, double* out) {
    if (check_args(N, Ci, H, W, K, border) || Co < 0) return 1;
    const int r = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        int64_t f = idx[t];
        int64_t c = f % Ci, pix = f / Ci;
        int64_t q = pix % W, p = (pix / W) % H, n = pix / (W * H);
        double sum = 0.0;
        for (int64_t i = p - r; i <= p + r; ++i) {
            if (i < 0 || i >= H) continue;
            for (int64_t j = q - r; j <= q + r; ++j) {
                if (j < 0 || j >= W) continue;
                const double* g = dy + ((n * H + i) * W + j) * Co;
                for (int a = 0; a < K; ++a) {
                    int64_t si;
                    if (!border_source(i + a - r, H, border, &si) || si != p) continue;
                    for (int b = 0; b < K; ++b) {
                        int64_t sj;
                        if (!border_source(j + b - r, W, border, &sj) || sj != q) continue;
                        for (int64_t o = 0; o < Co; ++o)
                            sum += w[((o * K + a) * (int64_t)K + b) * Ci + c] * g[o];
                    }
                }
            }
        }
        out[t] = sum;
    }
    return 0;
}

/* ------------------------------------------------------------- upsampling */

/* Nearest-neighbour upsampling by an integer factor s >= 1 (Section 4.2.3):
 * every pixel of the (H*s) x (W*s) output copies the input pixel found by
 * dividing its coordinates by s (integer division), plane by plane. */
int oracle_upsample_nearest(const double* x, double* y, int64_t planes, int64_t H, int64_t W,
                            int64_t s) {
    if (planes < 0 || H < 0 || W < 0 || s < 1) return 1;
    const int64_t Ho = H * s, Wo = W * s;
#pragma omp parallel for schedule(static)
    for (int64_t pl = 0; pl < planes; ++pl)
        for (int64_t p = 0; p < Ho; ++p)
            for (int64_t q = 0; q < Wo; ++q)
                y[(pl * Ho + p) * Wo + q] = x[(pl * H + p / s) * W + q / s];
    return 0;
}

/* The sharpening benchmark's output at selected flat NCHW indices of the
 * (N, C, H*s, W*s) result: the depthwise filter applied to the upsampled
 * image, with the border rule on the upsampled image.  The upsampled pixel
 * (u, v) is read as x[u / s][v / s], so the upsampled image is never built. */
int oracle_upsample_dw_fwd_points(const double* x, const double* w, int64_t N, int64_t C,
                                  int64_t H, int64_t W, int K, int border, int64_t s,
                                  const int64_t* idx, int64_t count, double* out) {
    if (check_args(N, C, H, W, K, border) || s < 1) return 1;
    const int64_t Ho = H * s, Wo = W * s;
    const int r = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        int64_t t = idx[k];
        const int64_t j = t % Wo; t /= Wo;
        const int64_t i = t % Ho; t /= Ho;
        const int64_t c = t % C, n = t / C;
        const double* plane = x + (n * C + c) * H * W;
        const double* f = w + c * (int64_t)K * K;
        double sum = 0.0;
        for (int a = 0; a < K; ++a) {
            int64_t su;
            if (!border_source(i + a - r, Ho, border, &su)) continue;
            for (int b = 0; b < K; ++b) {
                int64_t sv;
                if (!border_source(j + b - r, Wo, border, &sv)) continue;
                sum += f[a * K + b] * plane[(su / s) * W + sv / s];
            }
        }
        out[k] = sum;
    }
    return 0;
}

/* ------------------------------------------------------------- grayscale */

/* RGB to grayscale (Section 4.2.5): gray = 0.299 R + 0.587 G + 0.114 B per
 * pixel; x is N x 3 x H x W (channels R, G, B), gray is N x 1 x H x W. */
int oracle_rgb_to_gray(const double* x, double* gray, int64_t N, int64_t H, int64_t W) {
    if (N < 0 || H < 0 || W < 0) return 1;
    const int64_t P = H * W;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n)
        for (int64_t p = 0; p < P; ++p) {
            const double* px = x + n * 3 * P + p;
            gray[n * P + p] = 0.299 * px[0] + 0.587 * px[P] + 0.114 * px[2 * P];
        }
    return 0;
}
