"""GPU parity of the separable-filter path (a row pass then a column pass)
against the FP64 oracle -- the depthwise definition with the outer-product
filter -- through the C ABI, at sizes that span several tiles with ragged
tails, on both staging paths (W a multiple of 4: TMA; otherwise cp.async),
both borders and both storage types; and the benchmark-size image on sampled
outputs and every kind of border pixel.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import BF16_KERNEL_TOL, assert_fp32, normwise, poison_like, to_np

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
    wc = torch.randn((shape[1], K), generator=gen) * 0.3
    wr = torch.randn((shape[1], K), generator=gen) * 0.3
    return x.to(dtype), wc, wr


def fp32_check(y, x, wc, wr, border, K, what):
    b = BORDER[border]
    ref = oracle.dw_fwd_separable(x, wc, wr, b)
    mag = oracle.dw_fwd_separable(np.abs(x), np.abs(wc), np.abs(wr), b)
    # each output sums K row-pass values of K products each: bound with 2K terms
    assert_fp32(to_np(y), ref, mag, 2 * K, what)


@pytest.mark.parametrize("K", [1, 3, 5, 9, 15, 31])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("shape", [(2, 3, 67, 131), (1, 2, 130, 260), (1, 1, 5, 7),
                                   (1, 1, 1, 1)])
def test_separable_fp32(giga, K, border, shape):
    x, wc, wr = make(shape, K, 10 * K + shape[3])
    y = giga.conv2d_separable(x.cuda(), wc.cuda(), wr.cuda(), border,
                              out=poison_like(x.cuda()))
    fp32_check(y, x.numpy(), wc.numpy(), wr.numpy(), border, K, (shape, K, border))


@pytest.mark.parametrize("K", [3, 9])
@pytest.mark.parametrize("border", ["zero", "clamp"])
@pytest.mark.parametrize("W", [260, 264])
def test_separable_bf16(giga, K, border, W):
    x, wc, wr = make((2, 3, 67, W), K, 70 + K, torch.bfloat16)
    y = giga.conv2d_separable(x.cuda(), wc.cuda(), wr.cuda(), border)
    ref = oracle.dw_fwd_separable(x.double().numpy(), wc.numpy(), wr.numpy(), BORDER[border])
    assert normwise(to_np(y), ref) <= BF16_KERNEL_TOL


def test_separable_equals_full_filter_up_to_rounding(giga):
    """The separable path and the general K x K forward on the outer-product
    filter compute the same sums (different rounding order)."""
    x, wc, wr = make((1, 2, 200, 300), 7, 5)
    xc = x.cuda()
    ys = giga.conv2d_separable(xc, wc.cuda(), wr.cuda(), "clamp")
    yf = giga.conv2d_fwd(xc, (wc[:, :, None] * wr[:, None, :]).cuda(), "clamp")
    assert normwise(to_np(ys), to_np(yf)) < 2e-6


def test_gaussian_plain_small(giga):
    """512 x 512, the 5 x 5 normalised Gaussian (sigma 1) as its 1D factor,
    zero border: full compare."""
    x, w = workloads.plain_small()
    t = np.exp(-np.arange(-2, 3) ** 2 / 2.0)
    t = (t / t.sum()).astype(np.float32)
    f = torch.from_numpy(t)[None]
    y = giga.conv2d_separable(x.cuda(), f.cuda(), f.cuda(), "zero")
    ref = oracle.dw_fwd_separable(x.numpy(), t[None], t[None], oracle.ZERO)
    assert normwise(to_np(y), ref) <= 1e-5


@pytest.mark.parametrize("K", [3, 15])
def test_separable_at_scale_sampled(giga, K):
    """8 x 3 x 4096 x 4096 FP32, clamp border, as the benchmark runs it:
    sampled outputs and every kind of border pixel."""
    x, _ = workloads.plain_scale(K)
    gen = torch.Generator().manual_seed(900 + K)
    wc = torch.randn((3, K), generator=gen) * 0.3
    wr = torch.randn((3, K), generator=gen) * 0.3
    y = giga.conv2d_separable(x.cuda(), wc.cuda(), wr.cuda(), "clamp")
    N, C, H, W = x.shape
    idx = torch.unique(torch.cat([workloads.sample_indices(x.numel(), 2000, salt=50 + K),
                                  workloads.border_indices(N, C, H, W, per_plane=2,
                                                           salt=50 + K)]))
    got = y.reshape(-1)[idx.cuda()].double().cpu().numpy()
    wfull = (wc.double()[:, :, None] * wr.double()[:, None, :]).numpy()
    ref = oracle.dw_fwd_points(x.numpy(), wfull, oracle.CLAMP, idx.numpy())
    mag = oracle.dw_fwd_points(np.abs(x.numpy()), np.abs(wfull), oracle.CLAMP, idx.numpy())
    assert_fp32(got, ref, mag, 2 * K, ("scale", K))
    del y
    torch.cuda.empty_cache()
