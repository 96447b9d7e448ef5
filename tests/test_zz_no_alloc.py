"""The allocation-free filter gradient (giga_conv2d_bwd_filter_noalloc).

It exists for callers that cannot allocate device memory when they need the
gradient (a fixed memory budget, no workspace hook in their framework, or no
tolerance for cudaMalloc's implicit synchronisation); its partial sums live in
a scratch array inside the library.  These tests call it through the C ABI
and check it against giga_conv2d_bwd_filter with a caller-provided workspace.
The file is collected last on purpose, and each test also passes alone.
"""
import numpy as np
import pytest
import torch

from helpers import FP32_TOL, gamma, normwise, to_np


def _desc(lib, x, K, border):
    N, C, H, W = x.shape
    dt = lib.GIGA_F32 if x.dtype == torch.float32 else lib.GIGA_BF16
    return lib.desc(N, C, C, H, W, K, C, border, dt, lib.GIGA_LAYOUT_NCHW)


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
        x = torch.rand(shape, generator=gen).cuda()
        dy = torch.randn(shape, generator=gen).cuda()
        d = _desc(lib, x, K, border)
        ws_bytes = lib.giga_conv2d_workspace_size(d, lib.GIGA_OP_BWD_FILTER)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        ref = torch.empty((shape[1], K, K), device="cuda")
        mag = torch.empty((shape[1], K, K), device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        lib.check(lib.giga_conv2d_bwd_filter(d, x.data_ptr(), dy.data_ptr(), ref.data_ptr(),
                                             ws.data_ptr(), ws_bytes, s), "workspace version")
        # sum of |terms| per tap, for the elementwise FP32 bound
        ax, ady = x.abs(), dy.abs()
        lib.check(lib.giga_conv2d_bwd_filter(d, ax.data_ptr(), ady.data_ptr(), mag.data_ptr(),
                                             ws.data_ptr(), ws_bytes, s), "magnitudes")
        data.append((x, dy, d, ref, mag, K, shape))
    # two rounds of calls in a row; the scratch array keeps the previous
    # (different-sized) problem's partials between calls
    for _ in range(2):
        for x, dy, d, ref, mag, K, shape in data:
            out = torch.full((shape[1], K, K), float("nan"), device="cuda")
            st = lib.giga_conv2d_bwd_filter_noalloc(d, x.data_ptr(), dy.data_ptr(),
                                                    out.data_ptr(),
                                                    torch.cuda.current_stream().cuda_stream)
            lib.check(st, "giga_conv2d_bwd_filter_noalloc")
            torch.cuda.synchronize()
            o, r = to_np(out), to_np(ref)
            assert not np.isnan(o).any()
            # the parity tolerance: normwise 1e-5, and elementwise each side
            # within the FP32 bound of an n-term sum (so twice it between them)
            n = shape[0] * shape[2] * shape[3]
            assert normwise(o, r) <= FP32_TOL, (shape, K)
            assert (np.abs(o - r) <= 2 * gamma(n) * to_np(mag) + 1e-30).all(), (shape, K)


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
