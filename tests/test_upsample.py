"""GPU parity of nearest-neighbour upsampling (Section 4.2.3) and of the fused
upsample-then-filter pass (the sharpening benchmark, Section 6.6) against the
FP64 oracle, through the C ABI.

Small cases span several output tiles with ragged tails (upsampled sides not
multiples of the 64 x 128 tile, widths not multiples of 4), scales 1 to 20,
both borders and both storage types.  For K != 3 the fused pass must also
equal, bit for bit in FP32, the two-call path (upsample, then the depthwise
forward); for K = 3 the polyphase kernel adds the taps that land on one input
pixel before multiplying, so its FP32 bound counts K^2 + 4 rounded terms and
it is compared with the two-call path within that bound.  Every store width
of the polyphase kernel (16, 8, 4 bytes and scalar, FP32 and BF16, aligned and
offset outputs) is exercised.  The 4K-image workload is checked on sampled
outputs and on every kind of border pixel.
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


def n_terms(K, scale):
    """Rounded terms of one FP32 output: K^2 multiply-adds, or for the K = 3
    polyphase kernel (scale >= 2) up to 9 tap additions plus 4 multiply-adds."""
    return K * K + 4 if (K == 3 and scale > 1) else K * K


def make(shape, K, seed, dtype=torch.float32):
    gen = torch.Generator().manual_seed(seed)
    x = torch.rand(shape, generator=gen)
    w = torch.randn((shape[1], K, K), generator=gen) * 0.1
    return x.to(dtype), w


@pytest.mark.parametrize("shape,scale", [((2, 3, 13, 21), 1), ((1, 2, 13, 21), 2),
                                         ((1, 3, 9, 11), 3), ((1, 1, 7, 9), 5),
                                         ((1, 2, 3, 5), 20), ((1, 1, 1, 1), 7)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_upsample_nearest_exact(giga, shape, scale, dtype):
    x, _ = make(shape, 1, 11 + scale, dtype)
    y = giga.upsample_nearest(x.cuda(), scale, out=poison_like(
        torch.empty(shape[:2] + (shape[2] * scale, shape[3] * scale), dtype=dtype).cuda()))
    ref = oracle.upsample_nearest(x.double().numpy(), scale)
    assert np.array_equal(to_np(y), ref)


@pytest.mark.parametrize("K", [1, 3, 5, 7, 15])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("shape,scale", [((1, 2, 33, 45), 2), ((2, 1, 13, 21), 5),
                                         ((1, 3, 70, 97), 1), ((1, 1, 4, 6), 20)])
def test_upsample_conv2d_fp32(giga, K, border, shape, scale):
    x, w = make(shape, K, 100 * K + scale)
    xc, wc = x.cuda(), w.cuda()
    out_shape = shape[:2] + (shape[2] * scale, shape[3] * scale)
    y = giga.upsample_conv2d(xc, wc, scale, border,
                             out=poison_like(torch.empty(out_shape).cuda()))
    b = BORDER[border]
    ref = oracle.upsample_dw_fwd(x.numpy(), w.numpy(), b, scale)
    mag = oracle.upsample_dw_fwd(np.abs(x.numpy()), np.abs(w.numpy()), b, scale)
    assert_fp32(to_np(y), ref, mag, n_terms(K, scale), (shape, scale, K, border))
    up = giga.upsample_nearest(xc, scale)
    two = giga.conv2d_fwd(up, wc, border)
    if K == 3 and scale > 1:
        # polyphase: both within their bounds of the exact value
        assert_fp32(to_np(y), to_np(two), 2 * mag, n_terms(K, scale), (shape, scale, "two"))
    else:
        # the fused pass equals the two-call path bit for bit
        assert torch.equal(y, two), (shape, scale, K, border)


@pytest.mark.parametrize("scale", [2, 3, 4, 5, 6, 8, 16])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("hw", [(70, 37), (37, 70)])
def test_polyphase_store_widths(giga, scale, dtype, offset, border, hw):
    """The K = 3 polyphase kernel at every store width: s a multiple of 8, 4,
    2 or odd, FP32 and BF16, the output at an aligned address or one element
    past it (scalar stores), widths and heights that leave partial warps and
    items (W = 37: lanes past the image; H = 70: a second row group; W = 70,
    even: two input pixels per lane at s = 2, a partial second column block)."""
    shape = (1, 2) + hw
    x, w = make(shape, 3, 900 + scale + offset, dtype)
    out_shape = shape[:2] + (shape[2] * scale, shape[3] * scale)
    n_out = int(np.prod(out_shape))
    buf = torch.full((n_out + 8,), float("nan"), dtype=dtype).cuda()
    y = buf[offset:offset + n_out].view(out_shape)
    giga.upsample_conv2d(x.cuda(), w.cuda(), scale, border, out=y)
    b = BORDER[border]
    xd = x.double().numpy() if dtype == torch.bfloat16 else x.numpy()
    ref = oracle.upsample_dw_fwd(xd, w.numpy(), b, scale)
    if dtype == torch.float32:
        mag = oracle.upsample_dw_fwd(np.abs(x.numpy()), np.abs(w.numpy()), b, scale)
        assert_fp32(to_np(y), ref, mag, n_terms(3, scale), (scale, offset, border))
    else:
        assert normwise(to_np(y), ref) <= BF16_KERNEL_TOL
    # the guard elements around the output stay untouched
    assert torch.isnan(buf[:offset]).all() and torch.isnan(buf[offset + n_out:]).all()


@pytest.mark.parametrize("K", [3, 9])
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_upsample_conv2d_bf16(giga, K, border):
    shape, scale = (1, 3, 37, 52), 3
    x, w = make(shape, K, 500 + K, torch.bfloat16)
    y = giga.upsample_conv2d(x.cuda(), w.cuda(), scale, border)
    ref = oracle.upsample_dw_fwd(x.double().numpy(), w.numpy(), BORDER[border], scale)
    assert normwise(to_np(y), ref) <= BF16_KERNEL_TOL


def test_paper_laplacian_on_upsampled_constant(giga):
    """The paper's Laplacian (8 surrounded by -1) on an upsampled constant image
    is 0 wherever its window stays inside the image; under the clamp border it
    is 0 everywhere."""
    lap = torch.tensor([[[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]]).cuda()
    x = torch.full((1, 1, 50, 70), 0.75).cuda()
    y = giga.upsample_conv2d(x, lap, 4, "clamp")
    assert torch.count_nonzero(y).item() == 0
    y = giga.upsample_conv2d(x, lap, 4, "zero")
    assert torch.count_nonzero(y[..., 1:-1, 1:-1]).item() == 0


def test_invalid_scale_and_k(giga):
    from paper_2504_01266_gb300 import _lib
    x = torch.zeros((1, 1, 8, 8)).cuda()
    w = torch.zeros((1, 17, 17)).cuda()
    with pytest.raises(_lib.GigaError):
        giga.upsample_nearest(x, 0)
    with pytest.raises(_lib.GigaError):
        giga.upsample_conv2d(x, w, 2)


@pytest.mark.parametrize("scale", [2, 4, 8])
def test_4k_image_sampled(giga, scale):
    """A 3 x 2160 x 3840 image (the paper's 4K input) upsampled by 2, 4 and 8 and
    filtered with the paper's Laplacian, zero border, as the benchmark runs it:
    sampled outputs and every kind of border pixel."""
    gen = torch.Generator().manual_seed(2504 + 6)
    x = torch.rand((1, 3, 2160, 3840), generator=gen)
    lap = torch.tensor([[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]).repeat(3, 1, 1)
    y = giga.upsample_conv2d(x.cuda(), lap.cuda(), scale, "zero")
    N, C, Ho, Wo = y.shape
    idx = torch.cat([workloads.sample_indices(y.numel(), 3000, salt=scale),
                     workloads.border_indices(N, C, Ho, Wo, per_plane=2, salt=scale)])
    idx = torch.unique(idx)
    got = y.reshape(-1)[idx.cuda()].double().cpu().numpy()
    ref = oracle.upsample_dw_fwd_points(x.numpy(), lap.numpy(), oracle.ZERO, scale, idx.numpy())
    mag = oracle.upsample_dw_fwd_points(x.numpy(), np.abs(lap.numpy()), oracle.ZERO, scale,
                                        idx.numpy())
    assert_fp32(got, ref, mag, n_terms(3, scale), ("4k", scale))
    del y
    torch.cuda.empty_cache()
