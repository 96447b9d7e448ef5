"""Dense 3 x 3, 64 -> 64 channel filtering on tcgen05 (BF16 NHWC, FP32
accumulation, zero border) against the FP64 oracle on the BF16-rounded inputs,
through the C ABI.  Small cases span several 128-pixel tiles and a ragged
tail; the 8 x 1024 x 1024 x 64 workload is checked on sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import BF16_KERNEL_TOL, FP32_TOL, gamma, normwise, to_np


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def make(N, H, W, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.rand((N, H, W, 64), generator=g).to(torch.bfloat16)
    w = (torch.randn((64, 3, 3, 64), generator=g) * 0.05).to(torch.bfloat16)
    dy = torch.randn((N, H, W, 64), generator=g).to(torch.bfloat16)
    return x, w, dy


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 5, 200), (1, 9, 128), (1, 3, 300)])
def test_dense_fwd_and_input_grad(giga, shape):
    N, H, W = shape
    x, w, dy = make(N, H, W, sum(shape))
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    y = giga.dense_conv2d_fwd(xc, wc, out=torch.full_like(xc, float("nan")))
    dx = giga.dense_conv2d_bwd_input(dyc, wc, out=torch.full_like(dyc, float("nan")))
    giga.check_device_error()
    xr, wr, dyr = x.double().numpy(), w.double().numpy(), dy.double().numpy()
    assert normwise(to_np(y), oracle.dense_fwd(xr, wr, oracle.ZERO)) <= BF16_KERNEL_TOL
    assert normwise(to_np(dx), oracle.dense_bwd_input(dyr, wr, oracle.ZERO)) <= BF16_KERNEL_TOL


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 5, 200), (1, 3, 300), (3, 17, 64),
                                   (1, 4, 62), (1, 4, 63), (2, 3, 128), (1, 2, 191)])
def test_dense_filter_grad(giga, shape):
    """dw[o][a][b][c] = sum_{n,i,j} dy[n,i,j,o] x~[n,i+a-1,j+b-1,c] on the tensor
    cores (FP32 accumulation), FP64 across CTAs.  Bound: the FP32 accumulation
    bound 2 * gamma(n) * sum|terms| with n = N*H*W products per tap."""
    N, H, W = shape
    x, w, dy = make(N, H, W, 7 + sum(shape))
    dw = giga.dense_conv2d_bwd_filter(x.cuda(), dy.cuda(),
                                      out=torch.full((64, 3, 3, 64), float("nan"), device="cuda"))
    giga.check_device_error()
    xr, dyr = x.double().numpy(), dy.double().numpy()
    ref = oracle.dense_bwd_filter(xr, dyr, 3, oracle.ZERO)
    mag = oracle.dense_bwd_filter(np.abs(xr), np.abs(dyr), 3, oracle.ZERO)
    got = to_np(dw)
    assert not np.isnan(got).any()
    assert (np.abs(got - ref) <= 2 * gamma(N * H * W) * mag + 1e-30).all()
    assert normwise(got, ref) <= FP32_TOL


@pytest.mark.gpu
def test_dense_full_size_sampled(giga):
    """8 x 1024 x 1024 x 64 BF16, weights normal(0, 0.05): sampled outputs,
    including the image border, in the launch configuration the benchmark uses."""
    x, w, dy = workloads.dense()
    xc, wc = x.cuda(), w.cuda()
    y = giga.dense_conv2d_fwd(xc, wc)
    giga.check_device_error()
    idx = workloads.sample_indices(y.numel(), 4000, salt=5)
    edge = torch.tensor([((n * 1024 + i) * 1024 + j) * 64 + o
                         for n in (0, 7) for i in (0, 1023) for j in (0, 511, 1023)
                         for o in (0, 63)])
    idx = torch.unique(torch.cat([idx, edge]))
    got = y.reshape(-1)[idx.cuda()].double().cpu().numpy()
    ref = oracle.dense_fwd_points(x.double().numpy(), w.double().numpy(), oracle.ZERO,
                                  idx.numpy())
    assert normwise(got, ref) <= BF16_KERNEL_TOL


@pytest.mark.gpu
def test_dense_filter_grad_full_size_banded_dy(giga):
    """The filter gradient on the 8 x 1024 x 1024 x 64 workload in the launch
    configuration the benchmark uses, with dy zero outside two 8-row bands (in
    images 2 and 7): dw then equals the oracle's filter gradient of the
    10-row crops around the bands (the zero rows at the crop ends stand for the
    zero dy outside), so every CTA, chunk and the FP64 cross-CTA sum run at
    full size while the oracle works on 2 x 10 x 1024 pixels."""
    x, _, dy = workloads.dense()
    mask = torch.zeros((8, 1024, 1, 1), dtype=torch.bool)
    mask[2, 300:308] = True
    mask[7, 1016:1024] = True
    dyb = torch.where(mask, dy, torch.zeros_like(dy))
    dw = giga.dense_conv2d_bwd_filter(x.cuda(), dyb.cuda(),
                                      out=torch.full((64, 3, 3, 64), float("nan"), device="cuda"))
    giga.check_device_error()
    xs = torch.cat([x[2:3, 299:309], torch.cat([x[7:8, 1015:1024],
                                                torch.zeros_like(x[7:8, :1])], 1)]).double()
    dys = torch.cat([dyb[2:3, 299:309], torch.cat([dyb[7:8, 1015:1024],
                                                   torch.zeros_like(dyb[7:8, :1])], 1)]).double()
    ref = oracle.dense_bwd_filter(xs.numpy(), dys.numpy(), 3, oracle.ZERO)
    mag = oracle.dense_bwd_filter(np.abs(xs.numpy()), np.abs(dys.numpy()), 3, oracle.ZERO)
    got = to_np(dw)
    assert not np.isnan(got).any()
    assert (np.abs(got - ref) <= 2 * gamma(8 * 1024 * 1024) * mag + 1e-30).all()
    assert normwise(got, ref) <= FP32_TOL


def test_dense_rejects_unsupported():
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    a = 0x100000
    base = dict(N=1, C_in=64, C_out=64, H=8, W=8, K=3, groups=1, border=0,
                dtype=_lib.GIGA_BF16, layout=_lib.GIGA_LAYOUT_NHWC)
    for field, value, status in [("border", 1, _lib.GIGA_ERR_UNSUPPORTED),
                                 ("K", 5, _lib.GIGA_ERR_UNSUPPORTED),
                                 ("dtype", _lib.GIGA_F32, _lib.GIGA_ERR_UNSUPPORTED),
                                 ("C_in", 32, _lib.GIGA_ERR_UNSUPPORTED)]:
        args = dict(base)
        args[field] = value
        if field == "C_in":
            args["C_out"] = 32
        d = _lib.desc(**args)
        assert _lib.giga_conv2d_fwd(d, a, 2 * a, 3 * a, None, 0, None) == status, field
    d = _lib.desc(**base)
    assert _lib.giga_conv2d_fwd(d, a + 8, 2 * a, 3 * a, None, 0, None) == _lib.GIGA_ERR_MISALIGNED
