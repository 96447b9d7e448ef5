"""Autograd: the DepthwiseConv2d function's gradients (GPU, FP32) against FP64
central finite differences of L(x, w) = <conv(x, w), dy> computed with the
oracle on 64 x 64 crops, and against the oracle's own gradients.  L is
bilinear, so the FP64 central difference is exact up to rounding."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import FP32_TOL, normwise, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_autograd_matches_finite_differences(giga, border):
    # a 64 x 64 crop of the training workload (x uniform, 7 x 7 filters, dy normal)
    x, w, dy = workloads.train(N=2, C=3, H=64, W=64, K=7)
    b = oracle.ZERO if border == "zero" else oracle.CLAMP
    xc = x.cuda().requires_grad_(True)
    wc = w.cuda().requires_grad_(True)
    y = giga.conv2d(xc, wc, border)
    y.backward(dy.cuda())
    gx, gw = to_np(xc.grad), to_np(wc.grad)
    xn, wn, dyn = x.double().numpy(), w.double().numpy(), dy.double().numpy()

    def L(xx, ww):
        return float(np.vdot(oracle.dw_fwd(xx, ww, b), dyn))

    h = 1e-3
    g = np.random.default_rng(7)
    for _ in range(8):
        idx = tuple(int(v) for v in (g.integers(2), g.integers(3), g.integers(64), g.integers(64)))
        xp, xm = xn.copy(), xn.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (L(xp, wn) - L(xm, wn)) / (2 * h)
        assert abs(gx[idx] - fd) <= 1e-5 * max(1.0, np.abs(gx).max()), (idx, gx[idx], fd)
    for _ in range(8):
        idx = tuple(int(v) for v in (g.integers(3), g.integers(7), g.integers(7)))
        wp, wm = wn.copy(), wn.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (L(xn, wp) - L(xn, wm)) / (2 * h)
        assert abs(gw[idx] - fd) <= 1e-5 * max(1.0, np.abs(gw).max()), (idx, gw[idx], fd)
    # full gradients against the oracle's
    assert normwise(gx, oracle.dw_bwd_input(dyn, wn, b)) <= FP32_TOL
    assert normwise(gw, oracle.dw_bwd_filter(xn, dyn, 7, b)) <= FP32_TOL


def test_autograd_single_input_paths(giga):
    """Only one gradient requested: the function takes the unfused entry point."""
    x, w, dy = workloads.train(N=1, C=3, H=70, W=90, K=5)
    xc = x.cuda().requires_grad_(True)
    y = giga.conv2d(xc, w.cuda(), "clamp")
    y.backward(dy.cuda())
    assert normwise(to_np(xc.grad), oracle.dw_bwd_input(dy.numpy(), w.numpy(), 1)) <= FP32_TOL
    wc = w.cuda().requires_grad_(True)
    y = giga.conv2d(x.cuda(), wc, "clamp")
    y.backward(dy.cuda())
    assert normwise(to_np(wc.grad), oracle.dw_bwd_filter(x.numpy(), dy.numpy(), 5, 1)) <= FP32_TOL


def test_train_workload_sampled(giga):
    """16 x 3 x 2048 x 2048 FP32, 7 x 7, zero border: fused backward at full
    size, sampled input-gradient pixels and filter-gradient taps vs the oracle."""
    x, w, dy = workloads.train()
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    dx, dw = giga.conv2d_bwd(xc, dyc, wc, "zero")
    N, C, H, W = x.shape
    idx = torch.unique(torch.cat([workloads.sample_indices(x.numel(), 1500, salt=3),
                                  workloads.border_indices(2, C, H, W, per_plane=2, salt=3)]))
    got = dx.reshape(-1)[idx.cuda()].double().cpu().numpy()
    ref = oracle.dw_bwd_input_points(dy.numpy(), w.numpy(), 0, idx.numpy())
    assert normwise(got, ref) <= FP32_TOL
    taps = np.array([0, 24, 48, 49 + 10, 2 * 49 + 33])
    ref_dw = oracle.dw_bwd_filter_taps(x.numpy(), dy.numpy(), 7, 0, taps)
    got_dw = to_np(dw).reshape(-1)[taps]
    assert np.abs(got_dw - ref_dw).max() <= FP32_TOL * np.abs(ref_dw).max()
