// dense.cu -- the dense multi-channel 3 x 3 filter (C_in = C_out = 64, BF16
// NHWC, zero border) as an implicit GEMM on the 5th-generation tensor cores.
//
//   y[n][i][j][o] = sum_{a,b,c} w[o][a][b][c] * x[n][i + a - 1][j + b - 1][c]
//
// is, for each tile of 128 consecutive output pixels of one image row, a
// 128 x 64 x 576 GEMM: M = pixels, N = output channels, K = (tap, input
// channel).  The kernels here organise it around input-row bands: one TMA
// load brings 130 pixels of one input row (the tile plus its one-pixel halo;
// out-of-range pixels arrive as zeros, the zero border), and that band viewed
// from pixel b, times the weights of the three taps (0, b), (1, b), (2, b),
// is ONE MMA of N = 192 whose three 64-column blocks are the accumulators of
// the three output rows the band feeds.  The GigaAPI paper only remarks that
// convolution benefits from matrix multiplication (Section 3.1); this is that
// contraction done on tcgen05.
//
// Forward / input gradient: one persistent CTA per SM, 6 warps:
//   warp 0    TMA producer: all 9 weight taps once (72 KB, resident), then the
//             bands through a 6-slot ring;
//   warp 1    allocates 512 TMEM columns (a ring of 8 accumulators of 64
//             columns, one per output row) and one lane issues the MMAs
//             (3 pixel shifts x 4 K-steps of 16 per band);
//   warps 2-5 epilogue: tcgen05.ld of a finished row's accumulator (each warp
//             its 32-lane TMEM quadrant), re-zero it, convert to BF16, stage
//             the row swizzled in shared memory, one TMA store per tile.
// Operands are K-major with the 128-byte swizzle the TMA writes.  Every
// mbarrier wait is bounded: on expiry the CTA records an error code, stops
// issuing work and frees its TMEM (the host reads the code back).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace giga {

constexpr int kDenseC = 64;          // input and output channels
constexpr int kDenseTaps = 9;        // 3 x 3
constexpr int kDenseTileM = 128;     // output pixels per tile
constexpr int kDenseThreads = 192;
constexpr int kDenseABytes = kDenseTileM * kDenseC * 2;  // 16 KB
constexpr int kDenseBBytes = kDenseC * kDenseC * 2;      // 8 KB per tap
constexpr int kDenseTmemCols = 512;


// error codes written to *err (first one wins)
enum { kDenseErrNone = 0, kDenseErrTimeout = 1 };

// Barrier among the 4 epilogue warps only (named barrier 1, 128 threads).
__device__ __forceinline__ void epilogue_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
// The swizzle phase of each 128-byte row follows from its absolute shared
// address, so a start address 128 * b bytes into a 1024-aligned band (a view
// shifted by b pixels) needs no base offset.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// The same 128-byte-swizzled layout read as MN-major (the contiguous 128-byte
// rows hold 64 elements of M or N; consecutive rows step along K): 8-row K
// groups 1024 bytes apart, successive 64-element M/N blocks `lbo` bytes apart.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128,
// N = n (a multiple of 64 here).
__device__ __forceinline__ uint32_t kDenseIdescN(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}


__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          s_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_st16_zero(uint32_t taddr) {
  const uint32_t z = 0;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

__device__ __forceinline__ void tc_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct DenseParams {
  __nv_bfloat16* y;
  int* err;
  int N, H, W;
  int tiles_w;
  int64_t num_tiles;
};

__device__ __forceinline__ void dense_fail(int* err, volatile int* abort_flag) {
  atomicCAS(err, kDenseErrNone, kDenseErrTimeout);
  *abort_flag = 1;
}

// Work order: output-row tiles (n, strip jt, row i), i fastest; CTA b owns the
// contiguous range [b*T/G, (b+1)*T/G).  A run of consecutive rows i0 .. i1 - 1
// of one strip (at most kAccBufs rows, see run_end_of) needs input rows
// i0 - 1 .. i1 (130-pixel bands with the one-pixel halo on each side), each
// loaded once per run into a ring slot; output row i reads the bands
// of rows i - 1, i, i + 1, and tap (a, b) is the band of row i + a - 1 viewed
// from pixel b (a start address b * 128 bytes into the slot).
constexpr int kBandPx = kDenseTileM + 2;              // 130 pixels
constexpr int kBandBytes = kBandPx * kDenseC * 2;     // 16,640 bytes loaded
constexpr int kSlotBytes = 17 * 1024;                 // 1024-aligned slot
constexpr int kBandSlots = 6;
constexpr int kAccBufs = 8;                            // TMEM accumulators (64 columns each)
constexpr int kOutBufs = 2;                            // output staging tiles (16 KB each)
constexpr size_t kDenseSmemBand = 1024 + kDenseTaps * kDenseBBytes + kBandSlots * kSlotBytes +
                                  kOutBufs * kDenseABytes + 256;
static_assert((2 * kBandSlots + 2 + 2 * kAccBufs) * 8 + 4 <= 256, "barrier area");

__device__ __forceinline__ void tile_range(int64_t total, int64_t& begin, int64_t& end) {
  begin = total * blockIdx.x / gridDim.x;
  end = total * (blockIdx.x + 1) / gridDim.x;
}

// End of the run of output rows that starts at `tile`: a run stays inside one
// strip and inside one aligned group of kAccBufs rows in CTA order, so the
// rows any band touches own consecutive TMEM blocks and every MMA writes one
// contiguous column range.  (An MMA pair that straddled the end of the block
// ring ran at about 60 % of the rate of one contiguous MMA; the cost of the cap
// is two halo bands re-loaded, mostly from L2, per group of rows.)
__device__ __forceinline__ int64_t run_end_of(int64_t tile, int64_t t_begin, int64_t t_end, int H) {
  const int64_t strip_end = (tile / H + 1) * (int64_t)H;
  const int64_t group_end = t_begin + ((tile - t_begin) / kAccBufs + 1) * kAccBufs;
  return min(t_end, min(strip_end, group_end));
}

__global__ void __launch_bounds__(kDenseThreads, 1)
    dense_fwd_kernel(const __grid_constant__ CUtensorMap tmap_x,
                     const __grid_constant__ CUtensorMap tmap_w,
                     const __grid_constant__ CUtensorMap tmap_y, DenseParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sB = smem;
  uint8_t* sA = smem + kDenseTaps * kDenseBBytes;
  uint8_t* sOut = sA + kBandSlots * kSlotBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sOut + kOutBufs * kDenseABytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kBandSlots;
  uint64_t* bfull = bars + 2 * kBandSlots;
  uint64_t* tfull = bars + 2 * kBandSlots + 1;              // [kAccBufs]
  uint64_t* tempty = bars + 2 * kBandSlots + 1 + kAccBufs;  // [kAccBufs]
  uint64_t* drain = bars + 2 * kBandSlots + 1 + 2 * kAccBufs;  // the issuer's MMAs are done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ volatile int s_abort;
  __shared__ volatile int s_go;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t t_begin, t_end;
  tile_range(p.num_tiles, t_begin, t_end);

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kBandSlots; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(bfull, 1);
    for (int a = 0; a < kAccBufs; ++a) {
      mbar_init(tfull + a, 1);
      mbar_init(tempty + a, 4 * 32);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_addr(tmem_slot)),
                 "r"(kDenseTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      // taps are stored shift-major: slot (b * 3 + a), so the three taps of one
      // pixel shift b form one 192-row B operand
      mbar_expect_tx(bfull, kDenseTaps * kDenseBBytes);
      for (int t = 0; t < kDenseTaps; ++t)
        tma_load_2d(sB + ((t % 3) * 3 + t / 3) * kDenseBBytes, &tmap_w, t * kDenseC, 0, bfull);
      uint32_t seq = 0;  // global band-load counter: slot seq % S, phase (seq / S) & 1
      for (int64_t tile = t_begin; tile < t_end && !s_abort;) {
        // a run of rows of one strip: [tile, run_end)
        const int i0 = (int)(tile % p.H);
        const int64_t strip = tile / p.H;  // n * tiles_w + jt
        const int64_t run_end = run_end_of(tile, t_begin, t_end, p.H);
        const int i1 = i0 + (int)(run_end - tile);
        const int jt = (int)(strip % p.tiles_w);
        const int n = (int)(strip / p.tiles_w);
        for (int r = i0 - 1; r <= i1 && !s_abort; ++r, ++seq) {
          const int slot = (int)(seq % kBandSlots);
          if (!mbar_wait(empty + slot, ((seq / kBandSlots) & 1) ^ 1)) {
            dense_fail(p.err, &s_abort);
            break;
          }
          mbar_expect_tx(full + slot, kBandBytes);
          tma_load_4d(sA + slot * kSlotBytes, &tmap_x, 0, jt * kDenseTileM - 1, r, n, full + slot);
        }
        tile = run_end;
      }
      if (s_abort) {
        // let the loads still in flight land (bounded) before the CTA exits:
        // the weights and at most the last kBandSlots bands (an older band's
        // slot was refilled only after that band had arrived and been used)
        mbar_wait(bfull, 0);
        for (uint32_t q = seq > (uint32_t)kBandSlots ? seq - kBandSlots : 0; q < seq; ++q)
          mbar_wait(full + q % kBandSlots, (q / kBandSlots) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      // Band rho (an input row) with pixel shift b feeds output rows rho + 1,
      // rho, rho - 1 through taps a = 0, 1, 2: one MMA of N = 64 * (number of
      // those rows inside the run) into their accumulators.  Output row number
      // o (in CTA order) owns TMEM block acc_block(o) = R - 1 - (o mod R), so
      // rows o + 1, o, o - 1 sit in ascending blocks, contiguous because a run
      // never crosses a multiple of R in o.  Blocks arrive zeroed from the
      // epilogue; every MMA accumulates.
      bool ok = mbar_wait(bfull, 0);
      if (!ok) dense_fail(p.err, &s_abort);
      uint32_t seq = 0;   // band counter
      int64_t o_base = 0; // output-row number of the first row of the current run
      const uint32_t b_base = s_addr(sB);
      const uint32_t a_base = s_addr(sA);
      auto blk = [](int64_t o) { return kAccBufs - 1 - (int)(((o % kAccBufs) + kAccBufs) % kAccBufs); };
      for (int64_t tile = t_begin; ok && tile < t_end && !s_abort;) {
        const int64_t run_end = run_end_of(tile, t_begin, t_end, p.H);
        const int rows = (int)(run_end - tile);
        for (int k = 0; k < rows + 2 && ok; ++k) {
          // band k of the run is input row i0 - 1 + k; output row (run-local) k - 1
          const int64_t o_rho = o_base + k - 1;
          const int a_lo = (k - 1 + 1 <= rows - 1) ? 0 : ((k - 1 <= rows - 1) ? 1 : 2);
          const int a_hi = (k - 2 >= 0) ? 2 : ((k - 1 >= 0) ? 1 : 0);
          const uint32_t band = seq + k;
          if (!mbar_wait(full + band % kBandSlots, (band / kBandSlots) & 1)) {
            dense_fail(p.err, &s_abort);
            ok = false;
            break;
          }
          if (a_lo == 0) {
            // row o_rho + 1 is touched for the first time: its block must be free
            const int64_t o_new = o_rho + 1;
            if (!mbar_wait(tempty + blk(o_new), (uint32_t)((o_new / kAccBufs) & 1))) {
              dense_fail(p.err, &s_abort);
              ok = false;
              break;
            }
          }
          tc_fence_after();
          // the na rows sit in blocks q0 .. q0 + na - 1 <= kAccBufs - 1: a run
          // never leaves its aligned group of kAccBufs rows
          const int na = a_hi - a_lo + 1;
          const int q0 = blk(o_rho + 1 - a_lo);
          const uint32_t idesc = kDenseIdescN(64 * na);
          const uint32_t d_addr = tmem_base + (uint32_t)(q0 * 64);
          const uint32_t a_slot = a_base + (band % kBandSlots) * kSlotBytes;
#pragma unroll 1
          for (int b = 0; b < 3; ++b) {
            const uint32_t a_row = a_slot + b * 128;
            const uint32_t b_row = b_base + (b * 3 + a_lo) * kDenseBBytes;
#pragma unroll
            for (int kk = 0; kk < kDenseC / 16; ++kk)
              tc_mma(d_addr, sw128_desc(a_row + 32 * kk), sw128_desc(b_row + 32 * kk), idesc, 1u);
          }
          tc_commit(empty + band % kBandSlots);
          if (a_hi == 2) tc_commit(tfull + blk(o_rho - 1));  // row o_rho - 1 is complete
        }
        if (!ok) break;
        seq += rows + 2;
        o_base += rows;
        tile = run_end;
      }
      // every MMA issued above has completed before the CTA frees TMEM (at
      // once on the normal path, where the epilogue has waited for each row)
      tc_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // TMEM -> registers -> BF16 row of one pixel -> 128-byte-swizzled staging
    // tile in shared memory (conflict-free) -> one TMA tensor store per tile.
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    const int row = quad * 32 + lane;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    // every accumulator block starts zeroed (phase 0 of its "free" barrier)
    for (int q = 0; q < kAccBufs; ++q)
      for (int c = 0; c < 4; ++c) tc_st16_zero(lane_base + (uint32_t)(q * 64 + 16 * c));
    tc_wait_st();
    tc_fence_before();
    for (int q = 0; q < kAccBufs; ++q) mbar_arrive(tempty + q);
    int ob = 0;
    int64_t o = 0;  // output-row number in CTA order
    for (int64_t tile = t_begin; tile < t_end; ++tile, ++o) {
      const int q = kAccBufs - 1 - (int)(o % kAccBufs);
      const uint32_t par = (uint32_t)((o / kAccBufs) & 1);
      // The leader alone does the bounded waits and broadcasts the outcome, so
      // the four warps leave the loop together (they share a named barrier).
      if (leader) {
        int ok = !s_abort && mbar_wait(tfull + q, par);
        if (!ok) dense_fail(p.err, &s_abort);
        // staging buffer ob is free once the store issued from it two tiles
        // ago has finished reading it
        else bulk_wait_read<kOutBufs - 1>();
        s_go = ok;
      }
      epilogue_barrier();
      if (!s_go) break;
      tc_fence_after();
      const uint32_t taddr = lane_base + (uint32_t)(q * 64);
      float v[64];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float part[16];
        tc_ld16(taddr + 16 * c, part);
#pragma unroll
        for (int z = 0; z < 16; ++z) v[16 * c + z] = part[z];
      }
      tc_wait_ld();
      // hand the block back zeroed for the row o + R
#pragma unroll
      for (int c = 0; c < 4; ++c) tc_st16_zero(taddr + 16 * c);
      tc_wait_st();
      tc_fence_before();
      mbar_arrive(tempty + q);
      uint8_t* out_row = sOut + ob * kDenseABytes + row * 128;
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        uint4 u;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * z + 0], v[8 * z + 1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * z + 2], v[8 * z + 3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * z + 4], v[8 * z + 5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * z + 6], v[8 * z + 7]);
        u.x = *reinterpret_cast<uint32_t*>(&h0);
        u.y = *reinterpret_cast<uint32_t*>(&h1);
        u.z = *reinterpret_cast<uint32_t*>(&h2);
        u.w = *reinterpret_cast<uint32_t*>(&h3);
        // 128-byte swizzle: 16-byte chunk z of row r lives at chunk z ^ (r % 8)
        *reinterpret_cast<uint4*>(out_row + ((z ^ (row & 7)) << 4)) = u;
      }
      fence_proxy_async();
      epilogue_barrier();
      if (leader) {
        const int i = (int)(tile % p.H);
        const int64_t strip = tile / p.H;
        const int jt = (int)(strip % p.tiles_w);
        const int n = (int)(strip / p.tiles_w);
        tma_store_4d(&tmap_y, sOut + ob * kDenseABytes, 0, jt * kDenseTileM, i, n);
        bulk_commit();
      }
      ob ^= 1;
    }
    if (leader) bulk_wait_all();
  }

  // Drain: every MMA was waited for by the epilogue (tfull) before this point.
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kDenseTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------- filter gradient
//   dw[o][a][b][c] = sum_{n,i,j} dy[n][i][j][o] * x[n][i + a - 1][j + b - 1][c]
// Work unit: a chunk of 64 pixel positions k = 0..63 at j0 + k of one image
// row i.  A chunk needs three x bands (image rows i - 1, i, i + 1; pixels
// j0 - 1 .. j0 + 63, 65 pixels x 64 channels, one 128-byte row per pixel,
// 128-byte swizzle) and one dy band (row i, pixels j0 - 2 .. j0 + 63).  Both
// are read as MN-major operands (K = pixel position), a view b pixels into a
// band being a start address b * 128 bytes in (the swizzle phase follows the
// absolute shared address).  With A[k][c] = x[j0 + k - 1][c] (x band of tap
// row a, view 0) and B_s[k][o] = dy[j0 + k - s][o] (dy band, view 2 - s):
//   sum_k A[k][c] B_s[k][o] = sum_p x[p + s - 1][c] dy[p][o],  p = j0 + k - s,
// the contribution of tap (a, s) over the pixels p = j0 - s .. j0 + 63 - s.
// The chunks of a row (ceil((W + 2) / 64) of them) tile every pixel once for
// each s (dy is zero outside the image), so one MMA with N = 192 -- B = the
// three shifts s = 2, 1, 0 as 64-column N blocks 128 bytes apart -- gives all
// three taps of a filter row, and M = 128 stacks two filter rows (x bands of
// rows a and a + 1, one band slot apart):
//   MMA 0: rows a = 0, 1 -> 6 taps;   MMA 1: row a = 2 (the second M half,
//   band 2 viewed one pixel further, is computed and discarded).
// Chunks are ordered (image, column strip, row), row fastest, and CTA b owns
// a contiguous range of them, so consecutive chunks of a CTA walk down one
// column strip: each x band is loaded ONCE per run of rows into a ring of
// kWgXSlots slots and serves three chunks (rows i + 1, i, i - 1); dy bands go
// through their own ring.  MMA 0 needs the bands of rows i - 1 and i one slot
// apart: the band that lands in slot 0 is also written to a mirror slot after
// the last one, so the pair (last slot, slot 0) is adjacent too.  D
// accumulates in TMEM over all chunks of the CTA (2 x 192 columns); each CTA
// then writes its FP32 partial sums [tap][c][o] and a second kernel adds the
// CTAs' partials in FP64 in CTA order.
constexpr int kWgTileP = 64;                           // pixel positions per chunk (MMA K: 4 x 16)
constexpr int kWgXPx = kWgTileP + 1;                   // x band: 65 pixels
constexpr int kWgDyPx = kWgTileP + 2;                  // dy band: 66 pixels
constexpr int kWgSlot = 9 * 1024;                      // 1024-aligned band slots
constexpr int kWgXSlots = 12;                          // x ring (plus one mirror slot)
constexpr int kWgDySlots = 8;                          // dy ring
constexpr uint32_t kWgXTx = kWgXPx * kDenseC * 2;
constexpr uint32_t kWgDyTx = kWgDyPx * kDenseC * 2;
constexpr int kWgDyOff = (kWgXSlots + 1) * kWgSlot;
constexpr int kWgBarOff = kWgDyOff + kWgDySlots * kWgSlot;
constexpr int kWgN = 192;                              // three 64-channel shifts
constexpr int kWgTmemCols = 512;
constexpr size_t kWgSmem = 1024 + kWgBarOff + 512;
constexpr int64_t kWgPartialFloats = (int64_t)kDenseTaps * kDenseC * kDenseC;
static_assert(kWgSmem <= 227 * 1024, "filter-gradient shared memory");
static_assert((2 * kWgXSlots + 2 * kWgDySlots + 1) * 8 + 4 <= 512, "barrier area");

// M = 128, N = 192, both operands MN-major.
constexpr uint32_t kWgIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((uint32_t)(kWgN >> 3) << 17) | ((128u >> 4) << 24);

struct WgParams {
  float* partials;  // [grid][9][64][64]
  int* err;
  int N, H, W;
  int tiles_w;      // chunks per row: ceil((W + 2) / 64)
  int64_t num_tiles;
};

__global__ void __launch_bounds__(kDenseThreads, 1)
    dense_wgrad_kernel(const __grid_constant__ CUtensorMap tmap_x,
                       const __grid_constant__ CUtensorMap tmap_dy, WgParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sx = smem;                 // x slots 0 .. kWgXSlots (the last mirrors slot 0)
  uint8_t* sdy = smem + kWgDyOff;     // dy slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kWgBarOff);
  uint64_t* xfull = bars;
  uint64_t* xempty = bars + kWgXSlots;
  uint64_t* dyfull = bars + 2 * kWgXSlots;
  uint64_t* dyempty = bars + 2 * kWgXSlots + kWgDySlots;
  uint64_t* done = bars + 2 * kWgXSlots + 2 * kWgDySlots;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t t_begin, t_end;
  tile_range(p.num_tiles, t_begin, t_end);

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < kWgXSlots; ++q) {
      mbar_init(xfull + q, 1);
      mbar_init(xempty + q, 1);
    }
    for (int q = 0; q < kWgDySlots; ++q) {
      mbar_init(dyfull + q, 1);
      mbar_init(dyempty + q, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_addr(tmem_slot)),
                 "r"(kWgTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      // per run of rows i0 .. i1 - 1 of one strip: x bands i0 - 1 and i0, then
      // per chunk i the x band i + 1 and the dy band i (the MMA issuer's order)
      uint32_t xc = 0, dc = 0;  // x / dy band counters: slot c % S, phase (c / S) & 1
      for (int64_t tile = t_begin; tile < t_end && !s_abort;) {
        const int64_t strip = tile / p.H;  // n * tiles_w + jt
        const int64_t run_end = min(t_end, (strip + 1) * (int64_t)p.H);
        const int i0 = (int)(tile - strip * p.H);
        const int rows = (int)(run_end - tile);
        const int j0 = (int)(strip % p.tiles_w) * kWgTileP;
        const int n = (int)(strip / p.tiles_w);
        bool ok = true;
        for (int q = -1; q <= rows && ok && !s_abort; ++q) {
          // x band of image row i0 + q (rows -1 and H arrive as zeros)
          const int sl = (int)(xc % kWgXSlots);
          if (!(ok = mbar_wait(xempty + sl, ((xc / kWgXSlots) & 1) ^ 1))) break;
          mbar_expect_tx(xfull + sl, sl == 0 ? 2 * kWgXTx : kWgXTx);
          tma_load_4d(sx + sl * kWgSlot, &tmap_x, 0, j0 - 1, i0 + q, n, xfull + sl);
          if (sl == 0)
            tma_load_4d(sx + kWgXSlots * kWgSlot, &tmap_x, 0, j0 - 1, i0 + q, n, xfull + sl);
          ++xc;
          if (q < 1) continue;
          // dy band of image row i0 + q - 1 (its chunk needs x rows up to i0 + q)
          const int dl = (int)(dc % kWgDySlots);
          if (!(ok = mbar_wait(dyempty + dl, ((dc / kWgDySlots) & 1) ^ 1))) break;
          mbar_expect_tx(dyfull + dl, kWgDyTx);
          tma_load_4d(sdy + dl * kWgSlot, &tmap_dy, 0, j0 - 2, i0 + q - 1, n, dyfull + dl);
          ++dc;
        }
        if (!ok) {
          dense_fail(p.err, &s_abort);
          break;
        }
        tile = run_end;
      }
      if (s_abort) {
        // let the loads still in flight land (bounded) before the CTA exits:
        // at most the last kWgXSlots x bands and kWgDySlots dy bands
        for (uint32_t q = xc > (uint32_t)kWgXSlots ? xc - kWgXSlots : 0; q < xc; ++q)
          mbar_wait(xfull + q % kWgXSlots, (q / kWgXSlots) & 1);
        for (uint32_t q = dc > (uint32_t)kWgDySlots ? dc - kWgDySlots : 0; q < dc; ++q)
          mbar_wait(dyfull + q % kWgDySlots, (q / kWgDySlots) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      uint32_t xc = 0, dc = 0;  // same counters as the producer
      bool first = true, ok = true;
      const uint32_t x_base = s_addr(sx), dy_base = s_addr(sdy);
      auto wait_x = [&](uint32_t c) {
        return mbar_wait(xfull + c % kWgXSlots, (c / kWgXSlots) & 1);
      };
      for (int64_t tile = t_begin; ok && tile < t_end && !s_abort;) {
        const int64_t strip = tile / p.H;
        const int64_t run_end = min(t_end, (strip + 1) * (int64_t)p.H);
        const int rows = (int)(run_end - tile);
        ok = wait_x(xc) && wait_x(xc + 1);  // bands i0 - 1, i0
        for (int k = 0; ok && k < rows; ++k) {
          const uint32_t cb = xc + k;  // band of row i - 1 (i = i0 + k)
          const uint32_t cd = dc + k;
          if (!(ok = wait_x(cb + 2) &&
                     mbar_wait(dyfull + cd % kWgDySlots, (cd / kWgDySlots) & 1)))
            break;
          tc_fence_after();
          // MMA 0: bands i - 1 and i, one slot apart (the mirror after the last slot)
          const uint32_t a0 = x_base + (cb % kWgXSlots) * kWgSlot;
          // MMA 1: band i + 1 (second M half: the same band one pixel on, discarded)
          const uint32_t a1 = x_base + ((cb + 2) % kWgXSlots) * kWgSlot;
          const uint32_t b0 = dy_base + (cd % kWgDySlots) * kWgSlot;  // N block s' -> shift 2 - s'
#pragma unroll
          for (int kk = 0; kk < kWgTileP / 16; ++kk)
            tc_mma(tmem_base, sw128_desc_mn(a0 + kk * 2048, kWgSlot),
                   sw128_desc_mn(b0 + kk * 2048, 128), kWgIdesc, (first && kk == 0) ? 0u : 1u);
#pragma unroll
          for (int kk = 0; kk < kWgTileP / 16; ++kk)
            tc_mma(tmem_base + 256u, sw128_desc_mn(a1 + kk * 2048, 128),
                   sw128_desc_mn(b0 + kk * 2048, 128), kWgIdesc, (first && kk == 0) ? 0u : 1u);
          first = false;
          tc_commit(dyempty + cd % kWgDySlots);
          tc_commit(xempty + cb % kWgXSlots);  // band i - 1 has had its last use
        }
        if (!ok) {
          dense_fail(p.err, &s_abort);
          break;
        }
        // the run's last two bands (rows i1 - 1 and i1) are no longer needed
        tc_commit(xempty + (xc + rows) % kWgXSlots);
        tc_commit(xempty + (xc + rows + 1) % kWgXSlots);
        xc += rows + 2;
        dc += rows;
        tile = run_end;
      }
      // fires once every MMA issued above has completed (also after an abort,
      // so the epilogue's wait covers them before TMEM is freed)
      tc_commit(done);
    }
  } else {
    // epilogue: TMEM -> FP32 partials [tap][c][o] of this CTA.  TMEM lane
    // (row) = (half, c); MMA g, half h holds filter row a = 2g + h; column
    // block s' holds tap column b = 2 - s'.
    const int quad = warp & 3;
    const int half = quad >> 1, c = (quad & 1) * 32 + lane;
    const bool any = (int64_t)blockIdx.x < p.num_tiles;
    if (any && mbar_wait(done, 0) && !s_abort) {
      tc_fence_after();
      float* out = p.partials + (int64_t)blockIdx.x * kWgPartialFloats;
      for (int g = 0; g < 2; ++g) {
        const int a = 2 * g + half;
        for (int sb = 0; sb < 3; ++sb) {
          float v[64];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float part[16];
            tc_ld16(tmem_base + ((uint32_t)(quad * 32) << 16) +
                        (uint32_t)(g * 256 + sb * 64 + 16 * q),
                    part);
#pragma unroll
            for (int z = 0; z < 16; ++z) v[16 * q + z] = part[z];
          }
          tc_wait_ld();
          if (a < 3) {  // a == 3: the discarded half of MMA 1
            const int tap = 3 * a + (2 - sb);
            float4* dst = reinterpret_cast<float4*>(out + ((int64_t)tap * kDenseC + c) * kDenseC);
#pragma unroll
            for (int z = 0; z < 16; ++z)
              dst[z] = make_float4(v[4 * z], v[4 * z + 1], v[4 * z + 2], v[4 * z + 3]);
          }
        }
      }
    } else if (any) {
      dense_fail(p.err, &s_abort);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kWgTmemCols)
                 : "memory");
  }
}

// dw[o][a][b][c] = sum over CTAs (in order, FP64) of partial[cta][3a + b][c][o].
__global__ void dense_wgrad_finalize_kernel(const float* __restrict__ partials, int ctas,
                                            float* __restrict__ dw) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kDenseC * kDenseTaps * kDenseC) return;
  const int c = idx % kDenseC;
  const int tap = (idx / kDenseC) % kDenseTaps;
  const int o = idx / (kDenseC * kDenseTaps);
  double s = 0.0;
  for (int b = 0; b < ctas; ++b)
    s += (double)partials[(int64_t)b * kWgPartialFloats + ((int64_t)tap * kDenseC + c) * kDenseC + o];
  dw[idx] = (float)s;
}

// dgrad filter: wt[c][a][b][o] = w[o][2 - a][2 - b][c] (rotate the taps,
// swap the channel roles), so the input gradient is the same forward kernel
// run on dy.
__global__ void dense_flip_weights_kernel(const __nv_bfloat16* __restrict__ w,
                                          __nv_bfloat16* __restrict__ wt) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kDenseC * kDenseTaps * kDenseC) return;
  const int o = idx % kDenseC;
  const int tap = (idx / kDenseC) % kDenseTaps;
  const int c = idx / (kDenseC * kDenseTaps);
  const int a = tap / 3, b = tap % 3;
  wt[idx] = w[((o * 3 + (2 - a)) * 3 + (2 - b)) * kDenseC + c];
}

// ------------------------------------------------------------------ host
static __device__ int g_dense_err;

// The filter-gradient grid never exceeds this many CTAs (it is also capped by
// the SM count), so its workspace size does not depend on the device.
constexpr int kWgMaxCtas = 256;

size_t dense_workspace_bytes(bool input_grad) {
  return input_grad ? (size_t)(kDenseC * kDenseTaps * kDenseC * 2 + 255) / 256 * 256 : 0;
}

size_t dense_filter_workspace_bytes() {
  return (size_t)kWgMaxCtas * kWgPartialFloats * sizeof(float);
}

static bool make_nhwc_map(EncodeFn enc, CUtensorMap* m, const void* base, int64_t N, int64_t H,
                          int64_t W, int box_px) {
  cuuint64_t dims[4] = {(cuuint64_t)kDenseC, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
  cuuint64_t strides[3] = {(cuuint64_t)kDenseC * 2, (cuuint64_t)W * kDenseC * 2,
                           (cuuint64_t)H * W * kDenseC * 2};
  cuuint32_t box[4] = {(cuuint32_t)kDenseC, (cuuint32_t)box_px, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int device_sms() {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

// dw [64][3][3][64] FP32 = filter gradient of x, dy (NHWC BF16); ws holds the
// per-CTA partial sums (dense_filter_workspace_bytes()).
cudaError_t dense_wgrad_launch(const void* x, const void* dy, float* dw, int64_t N, int64_t H,
                               int64_t W, void* ws, cudaStream_t st) {
  EncodeFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tx, tdy;
  if (!make_nhwc_map(enc, &tx, x, N, H, W, kWgXPx) ||
      !make_nhwc_map(enc, &tdy, dy, N, H, W, kWgDyPx))
    return cudaErrorInvalidValue;
  int* err = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_dense_err);
  if (e != cudaSuccess) return e;
  e = set_smem_once<dense_wgrad_kernel>(kWgSmem);
  if (e != cudaSuccess) return e;
  WgParams prm;
  prm.partials = static_cast<float*>(ws);
  prm.err = err;
  prm.N = (int)N;
  prm.H = (int)H;
  prm.W = (int)W;
  prm.tiles_w = (int)((W + 2 + kWgTileP - 1) / kWgTileP);  // every pixel once for each shift
  prm.num_tiles = N * H * prm.tiles_w;
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(prm.num_tiles, device_sms()),
                                          kWgMaxCtas);
  dense_wgrad_kernel<<<grid, kDenseThreads, kWgSmem, st>>>(tx, tdy, prm);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int n = kDenseC * kDenseTaps * kDenseC;
  dense_wgrad_finalize_kernel<<<(n + 255) / 256, 256, 0, st>>>(prm.partials, grid, dw);
  note_launch();
  return cudaGetLastError();
}

// x [N][H][W][64] BF16, w [64][3][3][64] BF16 -> y [N][H][W][64] BF16.
// input_grad: x is dy, w is flipped into `ws` first, y is dx.
cudaError_t dense_launch(const void* x, const void* w, void* y, int64_t N, int64_t H, int64_t W,
                         bool input_grad, void* ws, cudaStream_t st) {
  EncodeFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const void* wk = w;
  if (input_grad) {
    const int n = kDenseC * kDenseTaps * kDenseC;
    dense_flip_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(
        static_cast<const __nv_bfloat16*>(w), static_cast<__nv_bfloat16*>(ws));
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wk = ws;
  }
  CUtensorMap tx, tw, ty;
  if (!make_nhwc_map(enc, &tx, x, N, H, W, kBandPx) ||
      !make_nhwc_map(enc, &ty, y, N, H, W, kDenseTileM))
    return cudaErrorInvalidValue;
  {
    cuuint64_t dims[2] = {(cuuint64_t)kDenseTaps * kDenseC, (cuuint64_t)kDenseC};
    cuuint64_t strides[1] = {(cuuint64_t)kDenseTaps * kDenseC * 2};
    cuuint32_t box[2] = {(cuuint32_t)kDenseC, (cuuint32_t)kDenseC};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(wk), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  int* err = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_dense_err);
  if (e != cudaSuccess) return e;
  e = set_smem_once<dense_fwd_kernel>(kDenseSmemBand);
  if (e != cudaSuccess) return e;
  DenseParams prm;
  prm.y = static_cast<__nv_bfloat16*>(y);
  prm.err = err;
  prm.N = (int)N;
  prm.H = (int)H;
  prm.W = (int)W;
  prm.tiles_w = (int)((W + kDenseTileM - 1) / kDenseTileM);
  prm.num_tiles = N * H * prm.tiles_w;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(prm.num_tiles, (int64_t)(sms > 0 ? sms : 148));
  dense_fwd_kernel<<<grid, kDenseThreads, kDenseSmemBand, st>>>(tx, tw, ty, prm);
  note_launch();
  return cudaGetLastError();
}

// Reads and clears the device error word of the dense kernels (synchronises
// the stream first).  Returns 0 or a kDenseErr* code.
cudaError_t dense_take_error(cudaStream_t st, int* code) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  int* err = nullptr;
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_dense_err);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(code, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpy(err, &zero, sizeof(int), cudaMemcpyHostToDevice);
}

}  // namespace giga
