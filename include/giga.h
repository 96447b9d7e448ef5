/*
 * giga.h -- C ABI of libgiga: dense 2D image filtering on one GB300 (sm_103a).
 *
 * The operation is the neighbourhood sum of the GigaAPI paper (Section 4.2.4,
 * "Sharpening"): every output pixel of every channel is the weighted sum of the
 * K x K neighbourhood centred on it, each neighbour multiplied by the filter
 * entry at the same offset from the filter centre (a cross-correlation; the
 * filter is not flipped).  Neighbours outside the image read zero (the paper
 * skips them: GIGA_BORDER_ZERO) or the nearest edge pixel, clamped per axis
 * (GIGA_BORDER_CLAMP).  With r = (K - 1) / 2 and the border rule applied to x:
 *
 *   depthwise (NCHW, w[C][K][K]):
 *     y[n][c][i][j] = sum_{a,b < K} w[c][a][b] * x[n][c][i + a - r][j + b - r]
 *   dense (NHWC, w[Co][K][K][Ci]):
 *     y[n][i][j][o] = sum_{a,b,c} w[o][a][b][c] * x[n][i + a - r][j + b - r][c]
 *
 * The gradients are the exact adjoints: dx = K^T dy (for the clamp border the
 * contributions that were read from clamped positions return to the edge pixel
 * they were read from) and dw[c][a][b] = sum_{n,i,j} dy[n][c][i][j] *
 * x[n][c][i + a - r][j + b - r] (the filter is shared by the batch, so the sum
 * runs over n).  The filter gradient is reduced in FP64 in a fixed order, so
 * repeated calls on the same device give bit-identical results.
 *
 * Conventions for every entry point:
 *   - Every pointer argument named x, y, dx, dy, w, dw, ws is a DEVICE pointer
 *     owned by the caller; no call allocates device memory and none keeps a
 *     pointer after it returns (batched plans keep host copies of their
 *     descriptors, see below).  The one piece of device memory the library
 *     holds is the fixed 4 MiB scratch array of
 *     giga_conv2d_bwd_filter_noalloc, which exists from the moment the
 *     library's code is loaded on a device until the process exits.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every launch is asynchronous on that stream; nothing synchronises the
 *     host unless stated.  The calls are safe to capture into a CUDA graph
 *     (the autotuner never benchmarks while the stream is capturing).
 *   - Argument errors are detected before any launch and return a status
 *     without touching memory; `giga_last_error_detail()` then describes the
 *     problem (thread-local).  A failed launch returns GIGA_ERR_CUDA.  No C++
 *     exception crosses this boundary.
 *   - Supported: odd K in [1, 31] (the filter gradient and the batched path:
 *     K <= 15); FP32 or BF16 storage for depthwise (weights, accumulation and
 *     dw always FP32); BF16 storage for dense (3 x 3, C_in = C_out = 64,
 *     zero border; dw FP32).  Tensors are dense and contiguous.
 *   - Inputs and outputs must not alias (y != x, dx != dy).
 */
#ifndef GIGA_H
#define GIGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t giga_status_t;
enum {
    GIGA_OK = 0,
    GIGA_ERR_INVALID_ARG = 1, /* bad shape, K, enum, NULL pointer or aliasing */
    GIGA_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. dense FP32)   */
    GIGA_ERR_MISALIGNED = 3,  /* pointer not aligned to its element size       */
    GIGA_ERR_WORKSPACE = 4,   /* workspace NULL, too small or not 256-B aligned */
    GIGA_ERR_CUDA = 5,        /* a CUDA call or launch failed                   */
    GIGA_ERR_TIMEOUT = 6      /* reserved: a bounded device wait gave up        */
};

enum { GIGA_BORDER_ZERO = 0, GIGA_BORDER_CLAMP = 1 };
enum { GIGA_F32 = 0, GIGA_BF16 = 1 };
enum { GIGA_LAYOUT_NCHW = 0, GIGA_LAYOUT_NHWC = 1 };
enum { GIGA_OP_FWD = 1, GIGA_OP_BWD_INPUT = 2, GIGA_OP_BWD_FILTER = 4 };

/* Problem descriptor (host memory, read during the call only).
 *   groups == C_in == C_out  -> depthwise, layout NCHW, dtype F32 or BF16
 *   groups == 1              -> dense, layout NHWC, dtype BF16
 * N, C, H, W may be 0 (nothing is launched; dw is zeroed). */
typedef struct {
    int64_t N, C_in, C_out, H, W;
    int32_t K;
    int32_t groups;
    int32_t border; /* GIGA_BORDER_* */
    int32_t dtype;  /* GIGA_F32 / GIGA_BF16: storage of x, y, dx, dy */
    int32_t layout; /* GIGA_LAYOUT_* */
    int32_t reserved; /* must be 0 */
} giga_conv2d_desc_t;

/* Bytes of device workspace the ops in `ops` (GIGA_OP_* bitmask) need for
 * this descriptor (Section 4.2.4's filter and the gradients derived from it;
 * only the filter gradient of the depthwise case and the dense gradients need
 * any).  0 means no workspace.  Workspaces must be 256-B aligned. */
giga_status_t giga_conv2d_workspace_size(const giga_conv2d_desc_t* desc, int32_t ops,
                                         size_t* bytes);

/* Forward filter (Section 4.2.4): y = K_w x.  Depthwise: x, y [N][C][H][W]
 * (dtype), w [C][K][K] FP32.  Dense: x [N][H][W][Ci], y [N][H][W][Co] BF16,
 * w [Co][K][K][Ci] BF16.  ws may be NULL when the size query returned 0. */
giga_status_t giga_conv2d_fwd(const giga_conv2d_desc_t* desc, const void* x, const void* w,
                              void* y, void* ws, size_t ws_bytes, void* stream);

/* Input gradient dx = K_w^T dy (same layouts as x / y): the adjoint of
 * Section 4.2.4's neighbourhood sum, every weighted read of the forward pass
 * sent back to the pixel it read (for the clamp border, the edge pixel the
 * clamped read landed on). */
giga_status_t giga_conv2d_bwd_input(const giga_conv2d_desc_t* desc, const void* dy,
                                    const void* w, void* dx, void* ws, size_t ws_bytes,
                                    void* stream);

/* Filter gradient dw = d<K_w x, dy>/dw, FP32, same layout as w: the
 * derivative of Section 4.2.4's neighbourhood sum with respect to each filter
 * entry, dw[c][a][b] = sum over n, i, j of dy[n][c][i][j] times the pixel tap
 * (a, b) reads for output (i, j).  Per-CTA FP32 partial sums go to the
 * workspace and are summed in FP64 in a fixed order. */
giga_status_t giga_conv2d_bwd_filter(const giga_conv2d_desc_t* desc, const void* x,
                                     const void* dy, float* dw, void* ws, size_t ws_bytes,
                                     void* stream);

/* Both gradients of Section 4.2.4's neighbourhood sum (the adjoint and the
 * filter derivative above) in one fused pass that reads x and dy once
 * (depthwise only; needs the workspace of GIGA_OP_BWD_INPUT |
 * GIGA_OP_BWD_FILTER). */
giga_status_t giga_conv2d_bwd(const giga_conv2d_desc_t* desc, const void* x, const void* dy,
                              const float* w, void* dx, float* dw, void* ws, size_t ws_bytes,
                              void* stream);

/* Filter gradient for callers that cannot allocate device memory.  The paper
 * has no counterpart: this serves code that runs under a fixed, pre-reserved
 * memory budget, plugins whose host framework offers no workspace, and paths
 * where cudaMalloc's implicit device synchronisation is not acceptable.
 * Arguments and result are those of giga_conv2d_bwd_filter without the
 * workspace: the per-CTA partial sums go to a scratch array inside the
 * library, a 4 MiB __device__ array (1,048,576 FP32 partial sums) that every
 * GPU which loads the library holds until the process exits.  The call itself
 * allocates nothing.
 *   - Limit: problems whose partial sums do not fit the array even with one
 *     CTA per image plane (N*C*K*K > 1,048,576) return GIGA_ERR_INVALID_ARG
 *     and say so in giga_last_error_detail(); use giga_conv2d_bwd_filter.
 *   - Chunking: the call starts from the chunk length giga_conv2d_bwd_filter
 *     would use (the autotuner's cached or pinned choice for this problem,
 *     else the built-in default; this entry point never benchmarks) and
 *     doubles it until the partial sums fit the array.  When no doubling is
 *     needed the result is bit-identical to giga_conv2d_bwd_filter's; when it
 *     is, the FP32 partials are grouped differently and the two agree to FP32
 *     rounding, not bit for bit.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress with that device current) and keeps it for the
 *     life of the process; make that first call before any stream capture.
 *     cudaDeviceReset invalidates the kept address: do not call this entry
 *     point on a device after resetting it.
 *   - All calls share the one array, which keeps the last call's contents
 *     (nothing in it needs to start at zero).  Calls that overlap on the GPU --
 *     different streams or host threads -- race on it; serialise them. */
giga_status_t giga_conv2d_bwd_filter_noalloc(const giga_conv2d_desc_t* desc, const void* x,
                                             const void* dy, float* dw, void* stream);

/* ------------------------------------------------------------------------
 * Ragged batches (the paper's unfinished "database of images", Section 5):
 * images of different sizes, each with its own depthwise filters, processed
 * by ONE persistent launch that pulls work from a tile table.
 *
 * One entry per image; all pointers are device pointers, NCHW with N = 1:
 *   x, y, dy, dx: [C][H][W] in the batch dtype; w, dw: [C][K][K] FP32.
 * Pointers of ops that are not requested may be NULL. */
typedef struct {
    const void* x;
    void* y;
    const void* dy;
    void* dx;
    const float* w;
    float* dw;
    int32_t H, W, C, K;
} giga_image_t;

typedef struct giga_batched_plan_s* giga_batched_plan_t;

/* Build the tile table on the host (sorted by cost, longest first).  `ops` is
 * a GIGA_OP_* bitmask; border and dtype apply to every image.  The plan copies
 * the descriptors; it owns host memory only. */
giga_status_t giga_batched_plan_create(const giga_image_t* images, int32_t n, int32_t ops,
                                       int32_t border, int32_t dtype,
                                       giga_batched_plan_t* plan);
giga_status_t giga_batched_plan_workspace_size(giga_batched_plan_t plan, size_t* bytes);
/* Copy the tile table into the workspace (asynchronous on `stream`; the plan
 * must outlive the copy -- giga_batched_plan_destroy waits for it). */
giga_status_t giga_batched_plan_upload(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                       void* stream);
/* One persistent launch for all images (plus a memset of its counters).
 * Capturable into a CUDA graph once the table has been uploaded.  `ws` must be
 * the workspace the current table was uploaded to (GIGA_ERR_WORKSPACE
 * otherwise); after a failed giga_batched_plan_autotune the plan refuses to
 * run (GIGA_ERR_INVALID_ARG) until it is uploaded again. */
giga_status_t giga_batched_plan_run(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                    void* stream);
void giga_batched_plan_destroy(giga_batched_plan_t plan);
/* Autotuner of the ragged launch (the paper has no tuner): times the
 * persistent launch with 1, 2, 4, 8, 16 and 32 tiles per chunk (a chunk is the
 * unit a CTA takes from the work counter; smaller chunks balance the tail,
 * larger ones cut the per-chunk reduction) on the caller's buffers -- the
 * outputs are overwritten -- then rebuilds and uploads the table for the
 * fastest.  Synchronises `stream`; not capturable
 * (GIGA_ERR_INVALID_ARG while the stream is capturing): call it before
 * capturing giga_batched_plan_run.  The plan's workspace size already covers
 * every candidate.  *tiles_per_chunk (may be NULL) receives the choice; the
 * default before any tuning is 4. */
giga_status_t giga_batched_plan_autotune(giga_batched_plan_t plan, void* ws, size_t ws_bytes,
                                         void* stream, int32_t* tiles_per_chunk);
/* Tiles per chunk the plan currently uses; -1 for a NULL plan. */
int32_t giga_batched_plan_tiles_per_chunk(giga_batched_plan_t plan);

/* Convenience: create + upload + run + destroy (blocks until the table copy
 * has left host memory; not capturable). */
giga_status_t giga_conv2d_batched(const giga_image_t* images, int32_t n, int32_t ops,
                                  int32_t border, int32_t dtype, void* ws, size_t ws_bytes,
                                  void* stream);
giga_status_t giga_conv2d_batched_workspace_size(const giga_image_t* images, int32_t n,
                                                 int32_t ops, size_t* bytes);

/* Separable depthwise filter: the K x K filter whose taps are
 * w[c][a][b] = wcol[c][a] * wrow[c][b] (wcol, wrow FP32 [C][K]), e.g. a
 * Gaussian or a box filter, applied as a row pass then a column pass in one
 * launch: 2K instead of K^2 multiply-adds per pixel.  Same tensors, layout,
 * borders and K range as giga_conv2d_fwd; the result equals giga_conv2d_fwd
 * with the outer-product filter up to rounding order (FP32 accumulation in
 * both passes).  Asynchronous on `stream`. */
giga_status_t giga_conv2d_fwd_separable(const giga_conv2d_desc_t* desc, const void* x,
                                        const float* wcol, const float* wrow, void* y,
                                        void* stream);

/* ------------------------------------------------------------------------
 * Upsampling (Section 4.2.3) and the sharpening benchmark (Section 6.6).
 * desc describes the INPUT: NCHW, N x C_in x H x W, groups == C_in ==
 * C_out, FP32 or BF16; the output y is N x C x (H * scale) x (W * scale) in
 * the same type, device memory owned by the caller, not aliasing x.
 *
 * giga_upsample_nearest: nearest-neighbour upsampling by the integer factor
 *   scale >= 1: y[n][c][p][q] = x[n][c][p / scale][q / scale] (integer
 *   division; every pixel becomes a scale x scale block).  desc->K and
 *   desc->border are checked but not used.
 * giga_upsample_conv2d_fwd: the depthwise K x K filter w[C][K][K] (FP32,
 *   odd K <= 15) applied to the upsampled image with desc->border on the
 *   upsampled image, in one pass: the upsampled image is never stored.
 *   Equal, bit for bit in FP32, to giga_upsample_nearest followed by
 *   giga_conv2d_fwd on its output.
 * Both are asynchronous on `stream`; GIGA_ERR_INVALID_ARG for scale < 1 or an
 * upsampled side of 2^31 or more. */
giga_status_t giga_upsample_nearest(const giga_conv2d_desc_t* desc, int32_t scale, const void* x,
                                    void* y, void* stream);
giga_status_t giga_upsample_conv2d_fwd(const giga_conv2d_desc_t* desc, int32_t scale,
                                       const void* x, const void* w, void* y, void* stream);

/* ------------------------------------------------------------------------
 * The sharpening benchmark over a ragged "database" of images (the batch
 * processing the paper gave up on, Section 5; the operation of Section 6.6
 * per image): every image is upsampled by its own integer scale and filtered
 * with its own depthwise filters.  All images of one filter size run in ONE
 * launch (at most 8 launches per batch, however many images it holds), each
 * CTA one output tile found through an image table in the workspace.
 *
 * One entry per image; device pointers, NCHW with N = 1:
 *   x: [C][H][W] and y: [C][H * scale][W * scale] in the batch dtype (not
 *   aliasing), w: [C][K][K] FP32.  Odd K <= 15 (GIGA_ERR_UNSUPPORTED above
 *   15), scale >= 2 (scale 1 is the plain filter: giga_conv2d_batched with
 *   GIGA_OP_FWD; GIGA_ERR_UNSUPPORTED), upsampled sides below 2^31.  Images
 *   with no output pixels are skipped.  The border rule applies on each
 *   upsampled image.  Every output equals giga_upsample_conv2d_fwd on that
 *   image alone, bit for bit.  `reserved` must be 0. */
typedef struct {
    const void* x;
    void* y;
    const float* w;
    int32_t H, W, C, K, scale;
    int32_t reserved;
} giga_up_image_t;

typedef struct giga_upsample_batched_plan_s* giga_upsample_batched_plan_t;

/* Build the image table on the host (images ordered by filter size, largest
 * first, then by size).  The plan copies the descriptors; it owns host memory
 * only.  The workspace (256-byte aligned) holds the table, which the kernels
 * only read. */
giga_status_t giga_upsample_batched_plan_create(const giga_up_image_t* images, int32_t n,
                                                int32_t border, int32_t dtype,
                                                giga_upsample_batched_plan_t* plan);
giga_status_t giga_upsample_batched_plan_workspace_size(giga_upsample_batched_plan_t plan,
                                                        size_t* bytes);
/* Copy the table into the workspace (asynchronous on `stream`; the plan must
 * outlive the copy -- giga_upsample_batched_plan_destroy waits for it). */
giga_status_t giga_upsample_batched_plan_upload(giga_upsample_batched_plan_t plan, void* ws,
                                                size_t ws_bytes, void* stream);
/* One launch per filter size present in the batch.  Capturable into a CUDA
 * graph once the table has been uploaded; `ws` must be the workspace it was
 * uploaded to (GIGA_ERR_WORKSPACE otherwise). */
giga_status_t giga_upsample_batched_plan_run(giga_upsample_batched_plan_t plan, void* ws,
                                             size_t ws_bytes, void* stream);
void giga_upsample_batched_plan_destroy(giga_upsample_batched_plan_t plan);

/* Convenience: create + upload + run + destroy (blocks until the table copy
 * has left host memory; not capturable). */
giga_status_t giga_upsample_conv2d_batched(const giga_up_image_t* images, int32_t n,
                                           int32_t border, int32_t dtype, void* ws,
                                           size_t ws_bytes, void* stream);
giga_status_t giga_upsample_conv2d_batched_workspace_size(const giga_up_image_t* images,
                                                          int32_t n, size_t* bytes);

/* ------------------------------------------------------------------------
 * Grayscale (Section 4.2.5): gray = 0.299 R + 0.587 G + 0.114 B per pixel.
 * desc: N images, C_in = 3 (channels R, G, B), C_out = 1, groups = 1, NCHW,
 * FP32 or BF16; x is N x 3 x H x W, y is N x 1 x H x W in the same type, not
 * aliasing x.
 * giga_rgb_to_gray: the conversion alone (desc->K, desc->border checked,
 *   not used).
 * giga_gray_conv2d_fwd: the K x K filter w[1][K][K] (FP32, odd K <= 15)
 *   applied to the gray image with desc->border, in one pass: the gray
 *   image is formed in shared memory and never stored.
 * Asynchronous on `stream`. */
giga_status_t giga_rgb_to_gray(const giga_conv2d_desc_t* desc, const void* x, void* y,
                               void* stream);
giga_status_t giga_gray_conv2d_fwd(const giga_conv2d_desc_t* desc, const void* x, const float* w,
                                   void* y, void* stream);

/* ------------------------------------------------------------------------
 * Autotuner.  Candidates: forward and input gradient (op 1 / 2): id 0..7 =
 * {8, 4} rows per thread (bit 0) x {one tile per CTA, persistent
 * double-buffered CTAs} (bit 1) x {no prefetch, an L2 prefetch of the tile
 * the CTA (or its successor) loads later} (bit 2); filter gradient (op 4): id 0..4 = tiles
 * per chunk of the persistent filter kernel {auto, 2, 4, 8, 16}; fused
 * backward (op 6): id 0..4 = the fused kernel with tiles per CTA {auto, 2,
 * 4, 8, 16}, id 5 = two passes (input gradient by the forward-style kernel
 * in the forward's tuned configuration, filter gradient by the filter
 * kernel), id 6 = one persistent kernel whose CTAs stream (x, dy) tile pairs
 * through a ring of two or three stages (the HBM-bound small filters).  The built-in default is id 0.
 * Modes (also from the environment variable GIGA_AUTOTUNE=off|cached|full):
 *   0 off:    always the built-in default configuration;
 *   1 cached: use a cached choice when one exists (default);
 *   2 full:   like cached, and the entry points benchmark the candidates the
 *             first time they meet an uncached problem class (not while the
 *             stream is capturing).
 * The cache is kept in memory and, if GIGA_AUTOTUNE_CACHE names a file,
 * loaded from / saved to it as JSON.  A corrupt cache file is ignored.  With
 * GIGA_LOG set (to anything but "0") every tuning decision, including the
 * ragged plan's, is printed to standard error with each candidate's time. */
giga_status_t giga_autotune_set_mode(int32_t mode);
int32_t giga_autotune_get_mode(void);
/* Benchmark every candidate for this problem on the given buffers (outputs
 * are overwritten; synchronises `stream`) and record the fastest. */
giga_status_t giga_autotune_conv2d(const giga_conv2d_desc_t* desc, int32_t ops, const void* x,
                                   const void* w, void* y, const void* dy, void* dx, float* dw,
                                   void* ws, size_t ws_bytes, void* stream);
/* The configuration id the entry points will use for (desc, op): the cached
 * choice, else 0; -1 on error. */
int32_t giga_autotune_choice(const giga_conv2d_desc_t* desc, int32_t op);
/* Pin configuration `id` for (desc's problem class, op) in the cache, as if
 * the tuner had chosen it; used in modes 1 and 2.  GIGA_ERR_INVALID_ARG for
 * an unknown op or an id outside the op's candidates. */
giga_status_t giga_autotune_set_choice(const giga_conv2d_desc_t* desc, int32_t op, int32_t id);
giga_status_t giga_autotune_save(const char* path);
giga_status_t giga_autotune_load(const char* path);
void giga_autotune_clear(void);

/* ------------------------------------------------------------------------ */
const char* giga_status_string(giga_status_t status);
/* Synchronise `stream`, then read and clear the device error words that the
 * kernels set when a bounded wait expires: the pipelined tensor-core kernels
 * (a barrier of their TMA / MMA pipeline) and the depthwise kernels (a TMA
 * tile load).  Such a kernel then stops issuing work, lets copies already in
 * flight land, releases its tensor memory and returns instead of hanging.
 * Returns GIGA_ERR_TIMEOUT if either word was set. */
giga_status_t giga_check_device_error(void* stream);
/* Failure-path self-test: launch one thread that waits on a barrier nothing
 * completes; its bounded wait gives up after 2 s and sets the depthwise error
 * word, so the next giga_check_device_error on the same stream returns
 * GIGA_ERR_TIMEOUT (and clears it).  Asynchronous; the device stays usable.
 * Not part of the paper's method: it exists to test failure detection. */
giga_status_t giga_selftest_bounded_wait(void* stream);
/* Description of the last error on the calling thread ("" if none). */
const char* giga_last_error_detail(void);
/* Kernel launches issued by this library on the calling thread since the last
 * reset (for launch accounting in benchmarks). */
uint64_t giga_launch_count(void);
void giga_launch_count_reset(void);

/* Measured FP32 multiply-add throughput of the current device, the
 * denominator of the ALU roofline of the depthwise kernels (not part of the
 * paper's method).  Runs 16 independent FMA chains per thread on every SM,
 * plain (packed = 0: fma.rn.f32) or packed (packed = 1: fma.rn.f32x2, two
 * FMAs per instruction): one warm-up launch, then the fastest of 5 timed
 * launches (CUDA events on `stream`; synchronises it; not capturable).
 * *tflops receives 2 x FMAs / time in TFLOP/s, *ms (may be NULL) that
 * launch's milliseconds.  `sink` is a device buffer of at least
 * giga_fp32_fma_peak_sink_bytes() bytes that receives one float per thread
 * (GIGA_ERR_WORKSPACE if smaller). */
size_t giga_fp32_fma_peak_sink_bytes(void);
giga_status_t giga_fp32_fma_peak(int32_t packed, float* sink, size_t sink_bytes, double* tflops,
                                 double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GIGA_H */
