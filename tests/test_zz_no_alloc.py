"""The allocation-free filter gradient (giga_conv2d_bwd_filter_noalloc).

It exists for callers that cannot allocate device memory when they need the
gradient (a fixed memory budget, no workspace hook in their framework, or no
tolerance for cudaMalloc's implicit synchronisation); its partial sums live in
a scratch array inside the library.  These tests call it through the C ABI
and check it against giga_conv2d_bwd_filter with a caller-provided workspace
and against the FP64 oracle.  The file is collected last on purpose, and each
test also passes alone.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_TOL, gamma, normwise, to_np


def _desc(lib, x, K, border):
    N, C, H, W = x.shape
    dt = lib.GIGA_F32 if x.dtype == torch.float32 else lib.GIGA_BF16
    return lib.desc(N, C, C, H, W, K, C, border, dt, lib.GIGA_LAYOUT_NCHW)


def _with_workspace(lib, d, x, dy, K):
    """giga_conv2d_bwd_filter with a workspace: dw and the same operator on
    |x|, |dy| (the sum of |terms| per tap, for the elementwise FP32 bound)."""
    C = x.shape[1]
    ws_bytes = lib.giga_conv2d_workspace_size(d, lib.GIGA_OP_BWD_FILTER)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ref = torch.empty((C, K, K), device="cuda")
    mag = torch.empty((C, K, K), device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    lib.check(lib.giga_conv2d_bwd_filter(d, x.data_ptr(), dy.data_ptr(), ref.data_ptr(),
                                         ws.data_ptr(), ws_bytes, s), "workspace version")
    ax, ady = x.abs(), dy.abs()
    lib.check(lib.giga_conv2d_bwd_filter(d, ax.data_ptr(), ady.data_ptr(), mag.data_ptr(),
                                         ws.data_ptr(), ws_bytes, s), "magnitudes")
    torch.cuda.synchronize()
    return ref, mag


def _noalloc(lib, d, x, dy, K):
    out = torch.full((x.shape[1], K, K), float("nan"), device="cuda")
    st = lib.giga_conv2d_bwd_filter_noalloc(d, x.data_ptr(), dy.data_ptr(), out.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    lib.check(st, "giga_conv2d_bwd_filter_noalloc")
    torch.cuda.synchronize()
    return out


@pytest.mark.gpu
def test_noalloc_matches_workspace_version_on_consecutive_calls():
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    lib = _lib
    gen = torch.Generator().manual_seed(2504)
    cases = [((2, 3, 67, 131), 7, lib.GIGA_BORDER_CLAMP),
             ((1, 3, 300, 500), 15, lib.GIGA_BORDER_ZERO),
             ((4, 2, 129, 256), 3, lib.GIGA_BORDER_CLAMP)]
    data = []
    for shape, K, border in cases:
        xh = torch.rand(shape, generator=gen)
        dyh = torch.randn(shape, generator=gen)
        x, dy = xh.cuda(), dyh.cuda()
        d = _desc(lib, x, K, border)
        ref, mag = _with_workspace(lib, d, x, dy, K)
        data.append((xh, dyh, x, dy, d, ref, mag, K, shape, border))
    # two rounds of calls in a row; the scratch array keeps the previous
    # (different-sized) problem's partials between calls
    for rnd in range(2):
        for xh, dyh, x, dy, d, ref, mag, K, shape, border in data:
            o, r = to_np(_noalloc(lib, d, x, dy, K)), to_np(ref)
            assert not np.isnan(o).any()
            # these partial sums fit the array at the workspace version's own
            # chunking, so the two runs are the same arithmetic
            assert np.array_equal(o, r), (shape, K)
            # the parity tolerance: normwise 1e-5, and elementwise each side
            # within the FP32 bound of an n-term sum (so twice it between them)
            n = shape[0] * shape[2] * shape[3]
            assert normwise(o, r) <= FP32_TOL, (shape, K)
            assert (np.abs(o - r) <= 2 * gamma(n) * to_np(mag) + 1e-30).all(), (shape, K)
            if rnd == 0:
                ob = oracle.CLAMP if border == lib.GIGA_BORDER_CLAMP else oracle.ZERO
                full = oracle.dw_bwd_filter(xh.numpy(), dyh.numpy(), K, ob)
                assert normwise(o, full) <= FP32_TOL, (shape, K)


@pytest.mark.gpu
def test_noalloc_doubles_chunks_to_fit_its_scratch():
    """A problem whose partial sums overflow the 1,048,576-float array at the
    chunk length the workspace version uses, but fit once it is doubled:
    64 planes of 2048 x 1024 (256 tiles each) at K = 15 with the tuner pinned
    to 2 tiles per chunk need 64 * 128 * 225 = 1,843,200 partials; at 4 tiles
    per chunk 921,600 fit."""
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    lib = _lib
    gen = torch.Generator().manual_seed(2505)
    shape, K = (1, 64, 2048, 1024), 15
    xh = torch.rand(shape, generator=gen)
    dyh = torch.randn(shape, generator=gen)
    x, dy = xh.cuda(), dyh.cuda()
    d = _desc(lib, x, K, lib.GIGA_BORDER_ZERO)
    mode = lib.giga_autotune_get_mode()
    try:
        lib.giga_autotune_set_mode(1)
        lib.check(lib.giga_autotune_set_choice(d, lib.GIGA_OP_BWD_FILTER, 1), "pin 2 tiles/chunk")
        ref, mag = _with_workspace(lib, d, x, dy, K)
        outs = [to_np(_noalloc(lib, d, x, dy, K)) for _ in range(2)]
    finally:
        lib.giga_autotune_clear()
        lib.giga_autotune_set_mode(mode)
    r = to_np(ref)
    n = shape[0] * shape[2] * shape[3]
    for o in outs:
        assert not np.isnan(o).any()
        assert normwise(o, r) <= FP32_TOL
        assert (np.abs(o - r) <= 2 * gamma(n) * to_np(mag) + 1e-30).all()
    # the fixed-order FP64 reduction makes repeated calls bit-identical
    assert np.array_equal(outs[0], outs[1])
    # sampled taps against the FP64 oracle (each a sum over 2M pixels)
    taps = np.array([0, 112, 224, 7 * 225 + 30, 31 * 225 + 200, 63 * 225 + 224])
    got = outs[0].reshape(-1)[taps]
    want = oracle.dw_bwd_filter_taps(xh.numpy().astype(np.float64),
                                     dyh.numpy().astype(np.float64), K, oracle.ZERO, taps)
    assert np.abs(got - want).max() <= FP32_TOL * np.abs(r).max()


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    lib = _lib
    # N*C*K*K = 100*64*225 = 1,440,000 partial sums > 1,048,576
    d = lib.desc(100, 64, 64, 64, 64, 15, 64, 0, lib.GIGA_F32, lib.GIGA_LAYOUT_NCHW)
    a = 0x100000
    st = lib.giga_conv2d_bwd_filter_noalloc(d, a, 2 * a, 3 * a, None)
    assert st == lib.GIGA_ERR_INVALID_ARG
    assert "too large" in lib.last_error_detail()
