"""GPU parity of the depthwise path against the FP64 oracle, through the C ABI.

Small cases span several tiles and ragged tails (H, W not multiples of the
64 x 128 tile, W not a multiple of 4, images smaller than the filter); the
full-size workloads are checked on sampled outputs and on every kind of
border pixel.  Outputs are poisoned with NaN first, so unwritten elements fail.
"""
import json
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import (BF16_E2E_TOL, BF16_KERNEL_TOL, FP32_TOL, assert_fp32, normwise,
                     poison_like, to_np)

pytestmark = pytest.mark.gpu

BORDER = {"zero": oracle.ZERO, "clamp": oracle.CLAMP}
SHAPES = [(2, 3, 67, 131), (1, 2, 130, 260), (1, 1, 8, 8), (1, 2, 5, 7), (1, 1, 1, 1),
          (2, 1, 3, 250), (1, 3, 200, 13)]
KS = [1, 3, 5, 7, 9, 11, 13, 15]


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def make(shape, K, seed, dtype=torch.float32):
    gen = torch.Generator().manual_seed(seed)
    x = torch.rand(shape, generator=gen)
    w = torch.randn((shape[1], K, K), generator=gen) * 0.1
    dy = torch.randn(shape, generator=gen)
    return x.to(dtype), w, dy.to(dtype)


@pytest.mark.parametrize("K", KS + [17, 31])
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_fwd_fp32(giga, K, border):
    for s, shape in enumerate(SHAPES):
        x, w, _ = make(shape, K, 100 * K + s)
        y = poison_like(x.cuda())
        giga.conv2d_fwd(x.cuda(), w.cuda(), border, out=y)
        b = BORDER[border]
        ref = oracle.dw_fwd(x.numpy(), w.numpy(), b)
        mag = oracle.dw_fwd(np.abs(x.numpy()), np.abs(w.numpy()), b)
        assert_fp32(to_np(y), ref, mag, K * K, (shape, K, border))


@pytest.mark.parametrize("K", [1, 3, 7, 15, 31])
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_bwd_input_fp32(giga, K, border):
    for s, shape in enumerate(SHAPES):
        _, w, dy = make(shape, K, 200 * K + s)
        dx = poison_like(dy.cuda())
        giga.conv2d_bwd_input(dy.cuda(), w.cuda(), border, out=dx)
        b = BORDER[border]
        ref = oracle.dw_bwd_input(dy.numpy(), w.numpy(), b)
        mag = oracle.dw_bwd_input(np.abs(dy.numpy()), np.abs(w.numpy()), b)
        # an edge pixel of the clamp fold sums up to (r + 1)^2 K^2 terms
        assert_fp32(to_np(dx), ref, mag, (K // 2 + 1) ** 2 * K * K, (shape, K, border))


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_bwd_fused_and_filter_fp32(giga, K, border):
    for s, shape in enumerate(SHAPES):
        x, w, dy = make(shape, K, 300 * K + s)
        xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
        dx, dw = giga.conv2d_bwd(xc, dyc, wc, border, dx=poison_like(dyc),
                                 dw=torch.full((shape[1], K, K), float("nan"), device="cuda"))
        dw_only = giga.conv2d_bwd_filter(xc, dyc, K, border)
        b = BORDER[border]
        ax, aw, ady = np.abs(x.numpy()), np.abs(w.numpy()), np.abs(dy.numpy())
        ref_dx = oracle.dw_bwd_input(dy.numpy(), w.numpy(), b)
        ref_dw = oracle.dw_bwd_filter(x.numpy(), dy.numpy(), K, b)
        assert_fp32(to_np(dx), ref_dx, oracle.dw_bwd_input(ady, aw, b),
                    (K // 2 + 1) ** 2 * K * K, (shape, K, border, "dx"))
        # each filter tap sums N*H*W products; the FP32 part of the reduction
        # sees at most that many terms, the cross-CTA part is FP64
        mag_dw = oracle.dw_bwd_filter(ax, ady, K, b)
        n = shape[0] * shape[2] * shape[3]
        assert_fp32(to_np(dw), ref_dw, mag_dw, n, (shape, K, border, "dw"))
        assert_fp32(to_np(dw_only), ref_dw, mag_dw, n, (shape, K, border, "dw only"))


@pytest.mark.parametrize("K", [3, 9, 15])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("shape", [(2, 3, 67, 260), (1, 2, 130, 264)])
def test_bf16(giga, K, border, shape):
    """BF16 storage: W = 260 rows (520 bytes) are staged by cp.async, W = 264
    rows (528 bytes, 16-byte multiple) by TMA."""
    x32, w, dy32 = make(shape, K, 400 + K)
    xb, dyb = x32.to(torch.bfloat16), dy32.to(torch.bfloat16)
    y = giga.conv2d_fwd(xb.cuda(), w.cuda(), border)
    dx, dw = giga.conv2d_bwd(xb.cuda(), dyb.cuda(), w.cuda(), border)
    b = BORDER[border]
    xr, dyr = xb.float().numpy(), dyb.float().numpy()   # the BF16-rounded inputs
    # (i) kernel error against the oracle on the rounded inputs
    assert normwise(to_np(y), oracle.dw_fwd(xr, w.numpy(), b)) <= BF16_KERNEL_TOL
    assert normwise(to_np(dx), oracle.dw_bwd_input(dyr, w.numpy(), b)) <= BF16_KERNEL_TOL
    assert normwise(to_np(dw), oracle.dw_bwd_filter(xr, dyr, K, b)) <= FP32_TOL
    # (ii) end to end against the oracle on the FP32 originals
    assert normwise(to_np(y), oracle.dw_fwd(x32.numpy(), w.numpy(), b)) <= BF16_E2E_TOL
    assert normwise(to_np(dx), oracle.dw_bwd_input(dy32.numpy(), w.numpy(), b)) <= BF16_E2E_TOL
    assert normwise(to_np(dw), oracle.dw_bwd_filter(x32.numpy(), dy32.numpy(), K, b)) \
        <= BF16_E2E_TOL


def test_plain_small_gaussian(giga):
    """512 x 512, one 5 x 5 normalised Gaussian (sigma 1), zero border: full compare."""
    x, w = workloads.plain_small()
    y = giga.conv2d_fwd(x.cuda(), w.cuda(), "zero")
    ref = oracle.dw_fwd(x.numpy(), w.numpy(), oracle.ZERO)
    assert normwise(to_np(y), ref) <= FP32_TOL


def test_filter_gradient_is_deterministic(giga):
    x, w, dy = make((4, 3, 300, 500), 7, 5)
    xc, dyc = x.cuda(), dy.cuda()
    a = giga.conv2d_bwd_filter(xc, dyc, 7, "clamp")
    b = giga.conv2d_bwd_filter(xc, dyc, 7, "clamp")
    assert torch.equal(a, b)


def test_misaligned_view_uses_scalar_path(giga):
    """A view starting one element in (not 16-byte aligned) takes the scalar
    staging path and still matches."""
    x, w, _ = make((1, 1, 40, 129), 5, 9)
    base = torch.zeros(40 * 129 + 1).cuda()
    base[1:] = x.reshape(-1).cuda()
    xv = base[1:].view(1, 1, 40, 129)
    y = giga.conv2d_fwd(xv, w.cuda(), "clamp")
    assert normwise(to_np(y), oracle.dw_fwd(x.numpy(), w.numpy(), oracle.CLAMP)) <= FP32_TOL


def _force_candidates(tmp_path, shape, K, border, dtype, choice):
    """Pin configurations through the autotune cache: choice maps the tuner's
    op index (0 forward, 1 input gradient, 2 filter gradient, 3 fused
    backward) to a candidate id; key: op, dtype, K, border, floor(log2(numel))."""
    from paper_2504_01266_gb300 import _lib
    N, C, H, W = shape
    dt = _lib.GIGA_F32 if dtype == torch.float32 else _lib.GIGA_BF16
    b = BORDER[border]
    sc = int(math.floor(math.log2(N * C * H * W)))
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"giga_autotune": 1, "entries": {
        f"{op}:{dt}:{K}:{b}:{sc}": cand for op, cand in choice.items()}}))
    _lib.giga_autotune_clear()
    assert _lib.giga_autotune_load(str(path)) == _lib.GIGA_OK
    d = _lib.desc(N, C, C, H, W, K, C, b, dt, _lib.GIGA_LAYOUT_NCHW)
    ops = {0: _lib.GIGA_OP_FWD, 1: _lib.GIGA_OP_BWD_INPUT, 2: _lib.GIGA_OP_BWD_FILTER,
           3: _lib.GIGA_OP_BWD_INPUT | _lib.GIGA_OP_BWD_FILTER}
    for op, cand in choice.items():
        assert _lib.giga_autotune_choice(d, ops[op]) == cand


class _CachedMode:
    def __enter__(self):
        from paper_2504_01266_gb300 import _lib
        self.mode = _lib.giga_autotune_get_mode()
        _lib.giga_autotune_set_mode(1)

    def __exit__(self, *exc):
        from paper_2504_01266_gb300 import _lib
        _lib.giga_autotune_clear()
        _lib.giga_autotune_set_mode(self.mode)


@pytest.mark.parametrize("K,border,dtype,W", [
    (3, "zero", torch.float32, 1000), (3, "clamp", torch.float32, 998),
    (15, "zero", torch.float32, 998), (15, "clamp", torch.float32, 1000),
    (7, "clamp", torch.float32, 1000), (3, "zero", torch.bfloat16, 1000),
    (15, "clamp", torch.bfloat16, 1000)])
def test_fwd_every_configuration(giga, tmp_path, K, border, dtype, W):
    """Every forward / input-gradient configuration ({8, 4} rows per thread x
    one tile per CTA or persistent double-buffered CTAs x with or without the
    L2 prefetch of a later tile) on planes holding
    more tiles than a persistent grid has CTAs, so each persistent CTA runs
    two or three tiles through its two shared-memory stages and the last
    round is ragged.  FP32 with W = 1000 is staged by TMA (the clamp border's
    edge tiles then fixed in shared memory), W = 998 by cp.async."""
    shape = (4, 4, 520, W)
    x, w, dy = make(shape, K, 600 + K, dtype)
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    b = BORDER[border]
    xr, dyr, wn = x.double().numpy(), dy.double().numpy(), w.numpy()
    ref_y, ref_dx = oracle.dw_fwd(xr, wn, b), oracle.dw_bwd_input(dyr, wn, b)
    if dtype == torch.float32:
        mag_y = oracle.dw_fwd(np.abs(xr), np.abs(wn), b)
        mag_dx = oracle.dw_bwd_input(np.abs(dyr), np.abs(wn), b)
    with _CachedMode():
        for cand in range(8):
            _force_candidates(tmp_path, shape, K, border, dtype, {0: cand, 1: cand})
            y = poison_like(xc)
            giga.conv2d_fwd(xc, wc, border, out=y)
            dx = poison_like(dyc)
            giga.conv2d_bwd_input(dyc, wc, border, out=dx)
            what = (K, border, dtype, cand)
            if dtype == torch.float32:
                assert_fp32(to_np(y), ref_y, mag_y, K * K, what)
                assert_fp32(to_np(dx), ref_dx, mag_dx, (K // 2 + 1) ** 2 * K * K, what)
            else:
                assert not torch.isnan(y).any() and not torch.isnan(dx).any(), what
                assert normwise(to_np(y), ref_y) <= BF16_KERNEL_TOL, what
                assert normwise(to_np(dx), ref_dx) <= BF16_KERNEL_TOL, what


@pytest.mark.parametrize("K,border,dtype,W", [
    (3, "clamp", torch.float32, 1000), (9, "zero", torch.float32, 998),
    (15, "clamp", torch.float32, 1000), (15, "zero", torch.float32, 1000),
    (5, "clamp", torch.float32, 998), (7, "zero", torch.bfloat16, 1000),
    (15, "clamp", torch.bfloat16, 1000)])
def test_bwd_every_configuration(giga, tmp_path, K, border, dtype, W):
    """Every filter-gradient configuration (tiles per chunk of the persistent
    filter kernel) and every fused-backward configuration (the fused kernel
    with each tiles-per-CTA choice, the two-pass split, and the persistent
    kernel with a two-stage tile ring) against the FP64 oracle.  16 planes of 520 x W hold 1152 tiles of 64 x 128: with 1 or 2
    tiles per chunk every persistent CTA runs several chunks back to back,
    so the shared-memory ring carries copies across chunk boundaries."""
    shape = (4, 4, 520, 998)
    x, w, dy = make(shape, K, 700 + K, dtype)
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    b = BORDER[border]
    xr, dyr, wn = x.double().numpy(), dy.double().numpy(), w.numpy()
    ref_dx = oracle.dw_bwd_input(dyr, wn, b)
    ref_dw = oracle.dw_bwd_filter(xr, dyr, K, b)
    mag_dx = oracle.dw_bwd_input(np.abs(dyr), np.abs(wn), b)
    mag_dw = oracle.dw_bwd_filter(np.abs(xr), np.abs(dyr), K, b)
    n = shape[0] * shape[2] * shape[3]
    nan_dw = lambda: torch.full((shape[1], K, K), float("nan"), device="cuda")

    def check_dw(dw, what):
        if dtype == torch.float32:
            assert_fp32(to_np(dw), ref_dw, mag_dw, n, what)
        else:   # FP32 accumulation of the BF16 inputs (exact products)
            assert normwise(to_np(dw), ref_dw) <= FP32_TOL, what

    def check_dx(dx, what):
        if dtype == torch.float32:
            assert_fp32(to_np(dx), ref_dx, mag_dx, (K // 2 + 1) ** 2 * K * K, what)
        else:
            assert not torch.isnan(dx).any(), what
            assert normwise(to_np(dx), ref_dx) <= BF16_KERNEL_TOL, what

    with _CachedMode():
        for cand in range(5):
            _force_candidates(tmp_path, shape, K, border, dtype, {2: cand})
            check_dw(giga.conv2d_bwd_filter(xc, dyc, K, border, out=nan_dw()),
                     (K, border, dtype, "filter", cand))
        for cand in range(7):
            _force_candidates(tmp_path, shape, K, border, dtype, {3: cand})
            dx, dw = giga.conv2d_bwd(xc, dyc, wc, border, dx=poison_like(dyc), dw=nan_dw())
            check_dx(dx, (K, border, dtype, "fused", cand))
            check_dw(dw, (K, border, dtype, "fused", cand))


# Shapes at the edges of the tiling: one image row of 2^20 pixels (TMA
# staging: 8,192 tile columns), the same with W % 4 = 3 (cp.async staging of
# unaligned rows), 2^20 + 1 rows of 3 pixels (16,385 tile rows of one
# partial column), and 65,537 planes of 4 x 4 (as many CTAs and filter
# channels, every tile mostly halo).
EXTREME = [((1, 1, 3, 1 << 20), 5), ((1, 1, 5, (1 << 20) + 3), 3),
           ((1, 1, (1 << 20) + 1, 3), 3), ((1, 65537, 4, 4), 3)]


@pytest.mark.parametrize("shape,K", EXTREME)
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_extreme_shapes(giga, shape, K, border):
    x, w, dy = make(shape, K, 1000 + K + shape[1] % 7)
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    b = BORDER[border]
    y = giga.conv2d_fwd(xc, wc, border, out=poison_like(xc))
    dx, dw = giga.conv2d_bwd(xc, dyc, wc, border, dx=poison_like(dyc),
                             dw=torch.full((shape[1], K, K), float("nan"), device="cuda"))
    torch.cuda.synchronize()
    xr, dyr, wn = x.double().numpy(), dy.double().numpy(), w.numpy()
    ax, ady, aw = np.abs(xr), np.abs(dyr), np.abs(wn)
    what = (shape, K, border)
    assert_fp32(to_np(y), oracle.dw_fwd(xr, wn, b), oracle.dw_fwd(ax, aw, b), K * K, what)
    assert_fp32(to_np(dx), oracle.dw_bwd_input(dyr, wn, b), oracle.dw_bwd_input(ady, aw, b),
                (K // 2 + 1) ** 2 * K * K, what)
    n = shape[0] * shape[2] * shape[3]
    assert_fp32(to_np(dw), oracle.dw_bwd_filter(xr, dyr, K, b),
                oracle.dw_bwd_filter(ax, ady, K, b), n, what)


# ------------------------------------------------------- full-size workloads

@pytest.mark.parametrize("K", [3, 7, 15])
def test_plain_scale_sampled(giga, K):
    """8 x 3 x 4096 x 4096 FP32, clamp border, in the benchmark's launch
    configuration; sampled outputs and every kind of border pixel."""
    x, w = workloads.plain_scale(K)
    xc, wc = x.cuda(), w.cuda()
    y = giga.conv2d_fwd(xc, wc, "clamp")
    N, C, H, W = x.shape
    idx = torch.cat([workloads.sample_indices(x.numel(), 3000, salt=K),
                     workloads.border_indices(N, C, H, W, per_plane=2, salt=K)])
    idx = torch.unique(idx)
    got = y.reshape(-1)[idx.cuda()].double().cpu().numpy()
    ref = oracle.dw_fwd_points(x.numpy(), w.numpy(), oracle.CLAMP, idx.numpy())
    assert normwise(got, ref) <= FP32_TOL
    del xc, y
    torch.cuda.empty_cache()


# The benchmark's tuned backward for 8 x 3 x 4096 x 4096 FP32 clamp: the fused
# kernel with 16 tiles per CTA at K = 3 (id 4) and automatic tiles per CTA at
# K = 7 (id 0); the two-pass split at K = 15 (id 5).
BENCH_BWD_CHOICE = {3: 4, 7: 0, 15: 5}


@pytest.mark.parametrize("K", [3, 7, 15])
def test_plain_scale_backward_sampled(giga, tmp_path, K):
    """8 x 3 x 4096 x 4096 FP32, clamp border, both gradients in the
    benchmark's tuned launch configuration: sampled dx pixels of the first and
    last image (edge rows and columns, where the clamp fold adds the margin
    sums, and the rows next to them included) and filter-gradient taps summed
    over the whole batch, against the oracle."""
    x, w = workloads.plain_scale(K)
    dy = workloads.plain_scale_dy()
    N, C, H, W = x.shape
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    with _CachedMode():
        _force_candidates(tmp_path, (N, C, H, W), K, "clamp", torch.float32,
                          {3: BENCH_BWD_CHOICE[K]})
        dx, dw = giga.conv2d_bwd(xc, dyc, wc, "clamp")
        torch.cuda.synchronize()
    del xc
    imgs = [0, N - 1]
    plane = C * H * W
    idx = torch.unique(torch.cat([
        workloads.sample_indices(2 * plane, 3000, salt=40 + K),
        workloads.border_indices(2, C, H, W, per_plane=2, salt=40 + K),
        torch.tensor([p * H * W + d * W + 777 for p in range(2 * C) for d in range(1, 9)] +
                     [p * H * W + 1234 * W + W - 1 - d for p in range(2 * C)
                      for d in range(1, 9)])]))
    full = torch.tensor(imgs)[idx // plane] * plane + idx % plane
    got = dx.reshape(-1)[full.cuda()].double().cpu().numpy()
    dy_sub = dy[imgs].numpy().astype(np.float64)
    ref = oracle.dw_bwd_input_points(dy_sub, w.numpy(), oracle.CLAMP, idx.numpy())
    assert normwise(got, ref) <= FP32_TOL
    kk = K * K
    taps = np.array([0, K - 1, kk // 2, kk - K, kk - 1, kk + 5, 2 * kk + kk // 3])
    ref_dw = oracle.dw_bwd_filter_taps(x.numpy().astype(np.float64),
                                       dy.numpy().astype(np.float64), K, oracle.CLAMP, taps)
    got_dw = to_np(dw).reshape(-1)[taps]
    assert np.abs(got_dw - ref_dw).max() <= FP32_TOL * np.abs(ref_dw).max()
    del dx, dw, dyc
    torch.cuda.empty_cache()


def test_bf16_workload_sampled(giga):
    """32 x 3 x 2048 x 2048 BF16 images, 9 x 9 filters, zero border -- the BF16
    comparison of the benchmark, in its launch configuration: sampled y and dx
    pixels (every kind of border pixel included) and a few filter-gradient taps
    against the oracle on the BF16-rounded inputs (kernel error) and on the
    FP32 originals (end to end)."""
    xb, w, dyb, x32, dy32 = workloads.bf16()
    xc, wc, dyc = xb.cuda(), w.cuda(), dyb.cuda()
    y = giga.conv2d_fwd(xc, wc, "zero")
    dx, dw = giga.conv2d_bwd(xc, dyc, wc, "zero")
    N, C, H, W = xb.shape
    idx = torch.unique(torch.cat([workloads.sample_indices(xb.numel(), 2000, salt=9),
                                  workloads.border_indices(2, C, H, W, per_plane=2, salt=9)]))
    ii = idx.numpy()
    xr, dyr = xb.float().numpy(), dyb.float().numpy()   # the BF16-rounded inputs
    for out, fn, a_r, a_32 in ((y, oracle.dw_fwd_points, xr, x32.numpy()),
                               (dx, oracle.dw_bwd_input_points, dyr, dy32.numpy())):
        got = out.reshape(-1)[idx.cuda()].double().cpu().numpy()
        assert normwise(got, fn(a_r, w.numpy(), oracle.ZERO, ii)) <= BF16_KERNEL_TOL
        assert normwise(got, fn(a_32, w.numpy(), oracle.ZERO, ii)) <= BF16_E2E_TOL
    taps = np.array([0, 40, 80, 81 + 17, 2 * 81 + 80])
    ref_dw = oracle.dw_bwd_filter_taps(xr, dyr, 9, oracle.ZERO, taps)
    got_dw = to_np(dw).reshape(-1)[taps]
    assert np.abs(got_dw - ref_dw).max() <= FP32_TOL * np.abs(ref_dw).max()
