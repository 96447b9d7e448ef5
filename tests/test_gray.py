"""GPU parity of RGB-to-grayscale (Section 4.2.5) and of the fused
grayscale-then-filter pass against the FP64 oracle, through the C ABI:
several tiles with ragged tails, both staging paths (W a multiple of 4: one
TMA load three planes deep; otherwise cp.async), both borders, both storage
types, and the equality of the fused pass with the two-call path (convert,
then the depthwise forward) bit for bit in FP32.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import BF16_KERNEL_TOL, FP32_TOL, assert_fp32, normwise, poison_like, to_np

pytestmark = pytest.mark.gpu

BORDER = {"zero": oracle.ZERO, "clamp": oracle.CLAMP}


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def make(shape, K, seed, dtype=torch.float32):
    gen = torch.Generator().manual_seed(seed)
    x = torch.rand(shape, generator=gen)
    w = torch.randn((1, K, K), generator=gen) * 0.1
    return x.to(dtype), w


@pytest.mark.parametrize("shape", [(2, 3, 67, 131), (1, 3, 130, 260), (1, 3, 1, 1)])
def test_rgb_to_gray(giga, shape):
    x, _ = make(shape, 1, shape[3])
    y = giga.rgb_to_gray(x.cuda())
    ref = oracle.rgb_to_gray(x.numpy())
    mag = oracle.rgb_to_gray(np.abs(x.numpy()))
    assert_fp32(to_np(y), ref, mag, 4, shape)


@pytest.mark.parametrize("K", [1, 3, 5, 9, 15])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("shape", [(2, 3, 67, 131), (1, 3, 130, 260), (1, 3, 5, 7)])
def test_gray_conv2d_fp32(giga, K, border, shape):
    x, w = make(shape, K, 30 * K + shape[2])
    xc, wc = x.cuda(), w.cuda()
    out = poison_like(torch.empty((shape[0], 1) + shape[2:]).cuda())
    y = giga.gray_conv2d(xc, wc, border, out=out)
    b = BORDER[border]
    ref = oracle.gray_dw_fwd(x.numpy(), w.numpy(), b)
    mag = oracle.gray_dw_fwd(np.abs(x.numpy()), np.abs(w.numpy()), b)
    # each output sums K^2 products of gray values, each a 3-term sum
    assert_fp32(to_np(y), ref, mag, K * K + 4, (shape, K, border))
    two = giga.conv2d_fwd(giga.rgb_to_gray(xc), wc, border)
    assert torch.equal(y, two), (shape, K, border)


@pytest.mark.parametrize("K", [3, 9])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("W", [260, 264])
def test_gray_conv2d_bf16(giga, K, border, W):
    x, w = make((2, 3, 67, W), K, 90 + K, torch.bfloat16)
    y = giga.gray_conv2d(x.cuda(), w.cuda(), border)
    ref = oracle.gray_dw_fwd(x.double().numpy(), w.numpy(), BORDER[border])
    assert normwise(to_np(y), ref) <= BF16_KERNEL_TOL


def test_gray_rejects_wrong_channels(giga):
    from paper_2504_01266_gb300 import _lib
    x = torch.zeros((1, 4, 8, 8)).cuda()
    with pytest.raises(ValueError):
        giga.gray_conv2d(x, torch.zeros((1, 3, 3)).cuda())
    d = _lib.desc(1, 4, 1, 8, 8, 3, 1, 0, _lib.GIGA_F32, _lib.GIGA_LAYOUT_NCHW)
    assert _lib.giga_gray_conv2d_fwd(d, x.data_ptr(), x.data_ptr(), x.data_ptr(), None) == \
        _lib.GIGA_ERR_INVALID_ARG


def test_gray_workload_full_size(giga):
    """8 RGB images of 4096 x 4096 FP32 with the paper's 3 x 3 Laplacian, zero
    border, in one launch as the benchmark runs it: images 0 and 7 compared
    with the oracle in full."""
    x, _ = workloads.plain_scale(3)   # read as R, G, B planes
    lap = torch.tensor([[[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]])
    y = giga.gray_conv2d(x.cuda(), lap.cuda(), "zero")
    for n in (0, 7):
        ref = oracle.gray_dw_fwd(x[n:n + 1].numpy(), lap.numpy(), oracle.ZERO)
        mag = oracle.gray_dw_fwd(x[n:n + 1].numpy(), np.abs(lap.numpy()), oracle.ZERO)
        assert_fp32(to_np(y[n:n + 1]), ref, mag, 9 + 4, ("image", n))
        assert normwise(to_np(y[n:n + 1]), ref) <= FP32_TOL
