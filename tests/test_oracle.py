"""Pins for the FP64 oracle, checked against facts the oracle does not compute
itself: hand-derived fixtures (tests/golden), closed forms, identities of the
mathematics, independent library routines (torch's FP64 CPU convolution and
nearest interpolation, numpy's repeat) and brute force on tiny inputs.  The
operation is the neighbourhood sum of the GigaAPI paper, Section 4.2.4
("Sharpening"), widened to K x K depthwise and dense filters, zero/clamp
borders and the two gradients, plus the nearest-neighbour upsampling of
Section 4.2.3 and the upsample-then-sharpen benchmark of Section 6.6.

Each ``pin_*`` function raises AssertionError when the oracle is wrong; the
pytest tests call them, and the mutation test at the bottom plants typical
mistakes in a copy of the oracle's C source and checks that some pin fails.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from golden_io import load as load_golden

ZERO, CLAMP = oracle.ZERO, oracle.CLAMP
BORDERS = {"zero": ZERO, "clamp": CLAMP}
pytestmark = pytest.mark.filterwarnings("ignore")


def rng(seed):
    return np.random.default_rng(2504 + seed)


def torch_dw(x, w, border):
    """Independent cross-check: torch's FP64 CPU conv2d (a cross-correlation)."""
    x = torch.as_tensor(x, dtype=torch.float64)
    w = torch.as_tensor(w, dtype=torch.float64)
    C, K = w.shape[0], w.shape[-1]
    r = (K - 1) // 2
    if border == ZERO:
        return F.conv2d(x, w[:, None], padding=r, groups=C).numpy()
    xp = F.pad(x, (r, r, r, r), mode="replicate")
    return F.conv2d(xp, w[:, None], groups=C).numpy()


def torch_dense(x_nhwc, w, border):
    x = torch.as_tensor(x_nhwc, dtype=torch.float64).permute(0, 3, 1, 2)
    wt = torch.as_tensor(w, dtype=torch.float64).permute(0, 3, 1, 2)  # (Co, Ci, K, K)
    r = (wt.shape[-1] - 1) // 2
    if border == ZERO:
        y = F.conv2d(x, wt, padding=r)
    else:
        y = F.conv2d(F.pad(x, (r, r, r, r), mode="replicate"), wt)
    return y.permute(0, 2, 3, 1).numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


SHAPES = [(1, 1, 8, 8), (2, 3, 9, 13), (1, 2, 5, 7), (1, 1, 1, 1), (1, 2, 2, 3), (2, 1, 16, 5)]
KS = [1, 3, 5, 7]


# ------------------------------------------------------------------ pins

def pin_golden():
    for name in ("paper_laplacian.txt", "shift_orientation.txt"):
        filt, cases = load_golden(name)
        for case, border, x, expect in cases:
            y = oracle.dw_fwd(x[None, None], filt[None], BORDERS[border])[0, 0]
            assert np.array_equal(y, expect), f"{name}:{case}\n{y}\n!=\n{expect}"


def pin_delta():
    for K in KS:
        for shape in SHAPES:
            x = rng(K).random(shape)
            w = np.zeros((shape[1], K, K)); w[:, K // 2, K // 2] = 1.0
            for b in (ZERO, CLAMP):
                assert np.array_equal(oracle.dw_fwd(x, w, b), x), (K, shape, b)


def pin_shift():
    """A one-hot filter at (a, b) moves the image by (a - r, b - r): closed form
    through numpy padding (constant for zero, edge replication for clamp)."""
    g = rng(1)
    for K in (3, 5):
        r = K // 2
        x = g.random((1, 1, 6, 9))
        for a in range(K):
            for b in range(K):
                w = np.zeros((1, K, K)); w[0, a, b] = 1.0
                for border, mode in ((ZERO, "constant"), (CLAMP, "edge")):
                    xp = np.pad(x[0, 0], r, mode=mode)
                    expect = xp[a:a + 6, b:b + 9]
                    y = oracle.dw_fwd(x, w, border)[0, 0]
                    assert np.array_equal(y, expect), (K, a, b, border)


def pin_box_constant():
    """Box filter 1/K^2 on a constant image c: clamp gives c everywhere, zero
    gives c * (in-image rows) * (in-image cols) / K^2."""
    c = 0.75
    for K in (3, 5, 7):
        r = K // 2
        for H, W in ((9, 11), (4, 3), (1, 6)):
            x = np.full((1, 1, H, W), c)
            w = np.full((1, K, K), 1.0 / (K * K))
            y = oracle.dw_fwd(x, w, CLAMP)
            assert np.allclose(y, c, rtol=1e-14, atol=0), (K, H, W)
            i = np.arange(H); j = np.arange(W)
            rows = np.minimum(i + r, H - 1) - np.maximum(i - r, 0) + 1
            cols = np.minimum(j + r, W - 1) - np.maximum(j - r, 0) + 1
            expect = c * rows[:, None] * cols[None, :] / (K * K)
            assert np.allclose(oracle.dw_fwd(x, w, ZERO)[0, 0], expect, rtol=1e-14, atol=0)


def pin_torch_crosscheck():
    g = rng(2)
    for K in KS + [9]:
        for shape in SHAPES:
            x = g.standard_normal(shape)
            w = g.standard_normal((shape[1], K, K))
            for border in (ZERO, CLAMP):
                assert rel(oracle.dw_fwd(x, w, border), torch_dw(x, w, border)) < 1e-13, \
                    (K, shape, border)


def pin_separable_gaussian():
    """A Gaussian K x K filter is the outer product of a 1D Gaussian: filtering
    with it equals a row-only pass followed by a column-only pass (holds for
    both borders because each axis is handled on its own)."""
    g = rng(3)
    for K in (3, 5, 7):
        r = K // 2
        t = np.exp(-np.arange(-r, r + 1) ** 2 / 2.0); t /= t.sum()
        full = np.outer(t, t)[None].repeat(2, 0)
        rowf = np.zeros((2, K, K)); rowf[:, r, :] = t
        colf = np.zeros((2, K, K)); colf[:, :, r] = t
        x = g.random((1, 2, 10, 12))
        for border in (ZERO, CLAMP):
            two = oracle.dw_fwd(oracle.dw_fwd(x, rowf, border), colf, border)
            assert rel(oracle.dw_fwd(x, full, border), two) < 1e-14, (K, border)


def pin_linearity():
    g = rng(4)
    x1, x2 = g.random((2, 3, 9, 10)), g.random((2, 3, 9, 10))
    w1, w2 = g.standard_normal((3, 5, 5)), g.standard_normal((3, 5, 5))
    for border in (ZERO, CLAMP):
        lhs = oracle.dw_fwd(2.0 * x1 - 3.0 * x2, w1, border)
        rhs = 2.0 * oracle.dw_fwd(x1, w1, border) - 3.0 * oracle.dw_fwd(x2, w1, border)
        assert rel(lhs, rhs) < 1e-13
        lhs = oracle.dw_fwd(x1, 0.5 * w1 + w2, border)
        rhs = 0.5 * oracle.dw_fwd(x1, w1, border) + oracle.dw_fwd(x1, w2, border)
        assert rel(lhs, rhs) < 1e-13


def pin_translation():
    """Shifting the image shifts the output wherever no border is involved."""
    g = rng(5)
    K, r = 5, 2
    x = g.random((1, 1, 20, 20))
    w = g.standard_normal((1, K, K))
    xs = np.roll(x, (3, 4), axis=(2, 3))
    y, ys = oracle.dw_fwd(x, w, ZERO), oracle.dw_fwd(xs, w, ZERO)
    # outputs whose window avoids the border and the wrapped region
    assert np.array_equal(ys[0, 0, 3 + r:20 - r, 4 + r:20 - r], y[0, 0, r:17 - r, r:16 - r])


def _operator_matrix(H, W, w, border):
    """Brute force: the columns of M are the images of the basis vectors."""
    n = H * W
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros((1, 1, H, W)); e.flat[k] = 1.0
        M[:, k] = oracle.dw_fwd(e, w, border).reshape(-1)
    return M


def pin_operator_bruteforce():
    """8 x 8 (and smaller, and K > image) operator matrices: M x equals the
    forward, M^T dy equals the input gradient, and the filter gradient equals
    the derivative of <M(w) x, dy> tap by tap."""
    g = rng(6)
    for (H, W, K) in ((8, 8, 3), (8, 8, 5), (5, 7, 3), (2, 3, 5), (1, 1, 3)):
        w = g.standard_normal((1, K, K))
        x = g.standard_normal((1, 1, H, W))
        dy = g.standard_normal((1, 1, H, W))
        for border in (ZERO, CLAMP):
            M = _operator_matrix(H, W, w, border)
            assert rel(oracle.dw_fwd(x, w, border).reshape(-1), M @ x.reshape(-1)) < 1e-13
            assert rel(oracle.dw_bwd_input(dy, w, border).reshape(-1),
                       M.T @ dy.reshape(-1)) < 1e-13, (H, W, K, border)
            dw = oracle.dw_bwd_filter(x, dy, K, border)
            for a in range(K):
                for b in range(K):
                    e = np.zeros((1, K, K)); e[0, a, b] = 1.0
                    Me = _operator_matrix(H, W, e, border)
                    expect = dy.reshape(-1) @ (Me @ x.reshape(-1))
                    assert abs(dw[0, a, b] - expect) <= 1e-12 * max(1.0, abs(expect))


def pin_adjoint():
    """<K x, y> = <x, K^T y> in FP64 for both borders, several K, ragged sizes."""
    g = rng(7)
    for K in (3, 7, 9):
        for shape in ((2, 3, 17, 23), (1, 2, 4, 31), (1, 1, 3, 2)):
            x, y = g.standard_normal(shape), g.standard_normal(shape)
            w = g.standard_normal((shape[1], K, K))
            for border in (ZERO, CLAMP):
                lhs = np.vdot(oracle.dw_fwd(x, w, border), y)
                rhs = np.vdot(x, oracle.dw_bwd_input(y, w, border))
                assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0), (K, shape, border)


def pin_filter_bilinear():
    """<K_w x, dy> = <w, G(x, dy)>: the filter gradient is the adjoint of the
    map w -> K_w x, summed over the whole batch."""
    g = rng(8)
    for K in (1, 3, 5, 7):
        for shape in ((3, 2, 11, 14), (1, 3, 5, 4)):
            x, dy = g.standard_normal(shape), g.standard_normal(shape)
            w = g.standard_normal((shape[1], K, K))
            for border in (ZERO, CLAMP):
                lhs = np.vdot(oracle.dw_fwd(x, w, border), dy)
                rhs = np.vdot(w, oracle.dw_bwd_filter(x, dy, K, border))
                assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0), (K, shape, border)


def pin_finite_differences():
    """L(x, w) = <conv(x, w), dy> is bilinear, so the FP64 central difference
    with h = 1e-3 is exact up to rounding: it must match both gradients."""
    g = rng(9)
    K, h = 7, 1e-3
    x = g.random((1, 3, 64, 64))
    w = g.normal(0, 0.1, (3, K, K))
    dy = g.standard_normal((1, 3, 64, 64))
    for border in (ZERO, CLAMP):
        L = lambda xx, ww: float(np.vdot(oracle.dw_fwd(xx, ww, border), dy))
        dx = oracle.dw_bwd_input(dy, w, border)
        pos = [(0, 0, 0), (1, 63, 63), (2, 0, 31), (0, 5, 63), (1, 32, 32), (2, 63, 1)]
        pos += [tuple(int(v) for v in (g.integers(3), g.integers(64), g.integers(64)))
                for _ in range(6)]
        for c, i, j in pos:
            xp, xm = x.copy(), x.copy()
            xp[0, c, i, j] += h; xm[0, c, i, j] -= h
            fd = (L(xp, w) - L(xm, w)) / (2 * h)
            assert abs(fd - dx[0, c, i, j]) <= 1e-8 * (1 + abs(fd)), (border, c, i, j)
        dw = oracle.dw_bwd_filter(x, dy, K, border)
        taps = [(0, 0, 0), (1, K - 1, K - 1), (2, 0, K - 1), (0, K // 2, K // 2)]
        taps += [tuple(int(v) for v in (g.integers(3), g.integers(K), g.integers(K)))
                 for _ in range(12)]
        for c, a, b in taps:
            wp, wm = w.copy(), w.copy()
            wp[c, a, b] += h; wm[c, a, b] -= h
            fd = (L(x, wp) - L(x, wm)) / (2 * h)
            assert abs(fd - dw[c, a, b]) <= 1e-8 * (1 + abs(fd)), (border, c, a, b)


def pin_points_match_full():
    g = rng(10)
    N, C, H, W, K = 2, 3, 13, 17, 5
    x, dy = g.standard_normal((N, C, H, W)), g.standard_normal((N, C, H, W))
    w = g.standard_normal((C, K, K))
    idx = g.choice(N * C * H * W, 200, replace=False)
    taps = g.choice(C * K * K, 20, replace=False)
    for border in (ZERO, CLAMP):
        assert np.array_equal(oracle.dw_fwd_points(x, w, border, idx),
                              oracle.dw_fwd(x, w, border).reshape(-1)[idx])
        assert rel(oracle.dw_bwd_input_points(dy, w, border, idx),
                   oracle.dw_bwd_input(dy, w, border).reshape(-1)[idx]) < 1e-13
        assert np.array_equal(oracle.dw_bwd_filter_taps(x, dy, K, border, taps),
                              oracle.dw_bwd_filter(x, dy, K, border).reshape(-1)[taps])


def pin_dense():
    """Dense case: torch cross-check, 1 x 1 channel reduces to depthwise, a
    channel-diagonal dense filter equals the depthwise one, both adjoints, and
    the point/tap evaluations equal the full ones."""
    g = rng(11)
    for (N, H, W, Ci, Co, K) in ((2, 6, 7, 3, 4, 3), (1, 5, 9, 2, 5, 5), (1, 1, 2, 3, 2, 3)):
        x = g.standard_normal((N, H, W, Ci))
        w = g.standard_normal((Co, K, K, Ci))
        dy = g.standard_normal((N, H, W, Co))
        for border in (ZERO, CLAMP):
            y = oracle.dense_fwd(x, w, border)
            assert rel(y, torch_dense(x, w, border)) < 1e-13, (N, H, W, Ci, Co, K, border)
            lhs = np.vdot(y, dy)
            assert abs(lhs - np.vdot(x, oracle.dense_bwd_input(dy, w, border))) \
                <= 1e-12 * (abs(lhs) + 1)
            assert abs(lhs - np.vdot(w, oracle.dense_bwd_filter(x, dy, K, border))) \
                <= 1e-12 * (abs(lhs) + 1)
            idx = g.choice(N * H * W * Co, min(50, N * H * W * Co), replace=False)
            assert np.array_equal(oracle.dense_fwd_points(x, w, border, idx), y.reshape(-1)[idx])
            dx = oracle.dense_bwd_input(dy, w, border)
            idx = g.choice(N * H * W * Ci, min(50, N * H * W * Ci), replace=False)
            assert rel(oracle.dense_bwd_input_points(dy, w, border, idx),
                       dx.reshape(-1)[idx]) < 1e-13
            dwf = oracle.dense_bwd_filter(x, dy, K, border)
            taps = g.choice(dwf.size, 10, replace=False)
            assert np.array_equal(oracle.dense_bwd_filter_taps(x, dy, K, border, taps),
                                  dwf.reshape(-1)[taps])
    # reductions to the depthwise operator
    x = g.standard_normal((2, 7, 8, 3))
    wd = g.standard_normal((3, 5, 5))
    wdense = np.zeros((3, 5, 5, 3))
    for c in range(3):
        wdense[c, :, :, c] = wd[c]
    for border in (ZERO, CLAMP):
        ref = oracle.dw_fwd(x.transpose(0, 3, 1, 2), wd, border).transpose(0, 2, 3, 1)
        assert rel(oracle.dense_fwd(x, wdense, border), ref) < 1e-14
        one = oracle.dense_fwd(x[..., :1], wd[:1, :, :, None], border)
        assert rel(one[..., 0], oracle.dw_fwd(x[..., :1].transpose(0, 3, 1, 2), wd[:1],
                                              border)[:, 0]) < 1e-14


def pin_upsample_nearest():
    """Nearest-neighbour upsampling (Section 4.2.3) against numpy's repeat and
    torch's FP64 nearest interpolation (both library routines), the identity at
    scale 1, and the structure of the result: constant s x s blocks whose
    stride-s subsampling gives back the input."""
    g = rng(21)
    for shape in [(1, 2, 5, 7), (2, 1, 3, 4), (1, 3, 1, 1)]:
        x = g.standard_normal(shape)
        assert np.array_equal(oracle.upsample_nearest(x, 1), x)
        for s in (2, 3, 5):
            up = oracle.upsample_nearest(x, s)
            assert up.shape == shape[:2] + (shape[2] * s, shape[3] * s)
            assert np.array_equal(up, np.repeat(np.repeat(x, s, axis=-2), s, axis=-1)), (shape, s)
            t = F.interpolate(torch.from_numpy(x), scale_factor=s, mode="nearest").numpy()
            assert np.array_equal(up, t), (shape, s)
            assert np.array_equal(up[..., ::s, ::s], x)
            for a in range(s):
                for b in range(s):
                    assert np.array_equal(up[..., a::s, b::s], x)


def pin_upsample_sharpen():
    """The sharpening benchmark (Section 6.6) = upsample, then filter: against
    torch's FP64 nearest interpolation followed by its FP64 depthwise
    convolution, and the point evaluations against the full arrays; the paper's
    Laplacian on an upsampled constant image is 0 wherever its 3 x 3 window
    stays inside the image."""
    g = rng(22)
    for K in (1, 3, 5):
        for s in (1, 2, 3):
            x = g.standard_normal((1, 2, 4, 6))
            w = g.standard_normal((2, K, K))
            xt = F.interpolate(torch.from_numpy(x), scale_factor=s, mode="nearest").numpy()
            for border in (ZERO, CLAMP):
                full = oracle.upsample_dw_fwd(x, w, border, s)
                assert rel(full, torch_dw(xt, w, border)) < 1e-13, (K, s, border)
                idx = np.arange(full.size)[::7]
                pts = oracle.upsample_dw_fwd_points(x, w, border, s, idx)
                assert np.array_equal(pts, full.reshape(-1)[idx]), (K, s, border)
    lap = np.array([[[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]])
    const = np.full((1, 1, 3, 5), 2.5)
    y = oracle.upsample_dw_fwd(const, lap, ZERO, 4)
    assert np.all(y[..., 1:-1, 1:-1] == 0.0)
    assert np.all(oracle.upsample_dw_fwd(const, lap, CLAMP, 4) == 0.0)


def pin_separable_filter():
    """A separable filter (column filter times row filter, both asymmetric and
    different) equals a row-only pass followed by a column-only pass, for both
    borders, and torch's FP64 convolution with the K x 1 then 1 x K kernels
    (zero border) -- which also fixes which factor runs along which axis."""
    g = rng(23)
    for K in (3, 5, 9):
        r = K // 2
        wc = g.standard_normal((2, K))
        wr = g.standard_normal((2, K))
        x = g.standard_normal((2, 2, 11, 13))
        rowf = np.zeros((2, K, K)); rowf[:, r, :] = wr
        colf = np.zeros((2, K, K)); colf[:, :, r] = wc
        for border in (ZERO, CLAMP):
            two = oracle.dw_fwd(oracle.dw_fwd(x, rowf, border), colf, border)
            assert rel(oracle.dw_fwd_separable(x, wc, wr, border), two) < 1e-13, (K, border)
        xt = torch.from_numpy(x)
        t = F.conv2d(xt, torch.from_numpy(wc)[:, None, :, None], padding=(r, 0), groups=2)
        t = F.conv2d(t, torch.from_numpy(wr)[:, None, None, :], padding=(0, r), groups=2)
        assert rel(oracle.dw_fwd_separable(x, wc, wr, ZERO), t.numpy()) < 1e-13, K
        assert rel(oracle.dw_fwd_separable(x, wr, wc, ZERO), t.numpy()) > 1e-3, K


def pin_grayscale():
    """Section 4.2.5's luminance weights: pure red, green and blue images give
    0.299, 0.587 and 0.114 times their value; equal channels give the value
    back (the weights sum to 1); the conversion equals the weighted channel sum
    computed by numpy and by torch, and composes with the filter."""
    g = rng(24)
    x = g.standard_normal((2, 3, 5, 7))
    want = 0.299 * x[:, 0] + 0.587 * x[:, 1] + 0.114 * x[:, 2]
    got = oracle.rgb_to_gray(x)
    assert got.shape == (2, 1, 5, 7)
    assert rel(got[:, 0], want) < 1e-15
    t = (torch.from_numpy(x) * torch.tensor([0.299, 0.587, 0.114], dtype=torch.float64)[:, None, None]).sum(1)
    assert rel(got[:, 0], t.numpy()) < 1e-15
    for ch, coef in enumerate((0.299, 0.587, 0.114)):
        pure = np.zeros((1, 3, 2, 2))
        pure[0, ch] = 2.0
        assert np.allclose(oracle.rgb_to_gray(pure), 2.0 * coef, rtol=1e-15, atol=0)
    same = np.repeat(x[:, :1], 3, axis=1)
    assert rel(oracle.rgb_to_gray(same), x[:, :1]) < 1e-15
    w = g.standard_normal((1, 3, 3))
    for border in (ZERO, CLAMP):
        assert rel(oracle.gray_dw_fwd(x, w, border),
                   oracle.dw_fwd(want[:, None], w, border)) < 1e-14


PINS = [pin_golden, pin_delta, pin_shift, pin_box_constant, pin_torch_crosscheck,
        pin_separable_gaussian, pin_linearity, pin_translation, pin_operator_bruteforce,
        pin_adjoint, pin_filter_bilinear, pin_finite_differences, pin_points_match_full,
        pin_dense, pin_upsample_nearest, pin_upsample_sharpen, pin_separable_filter,
        pin_grayscale]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_invalid_arguments_rejected():
    x = np.zeros((1, 1, 4, 4))
    with pytest.raises(ValueError):
        oracle.dw_fwd(x, np.zeros((1, 2, 2)), ZERO)          # even K
    with pytest.raises(ValueError):
        oracle.dw_fwd(x, np.zeros((1, 3, 3)), 7)             # unknown border


# ------------------------------------------------------- planted mistakes

# Each mutation rewrites one line of a copy of the oracle's C source.  The
# strings are matched exactly, so a refactor of the oracle that breaks a
# match fails loudly here instead of silently testing nothing.
MUTATIONS = {
    "convolution_not_correlation": (
        "sum += f[a * K + b] * plane[si * W + sj];",
        "sum += f[(K - 1 - a) * K + (K - 1 - b)] * plane[si * W + sj];"),
    "filter_transposed": (
        "sum += f[a * K + b] * plane[si * W + sj];",
        "sum += f[b * K + a] * plane[si * W + sj];"),
    "last_tap_dropped": (
        "sum += f[a * K + b] * plane[si * W + sj];",
        "sum += (b == K - 1 ? 0.0 : f[a * K + b]) * plane[si * W + sj];"),
    "clamp_reflects_low_edge": (
        "*src = p < 0 ? 0 : n - 1;",
        "*src = p < 0 ? (n > 1 ? 1 : 0) : n - 1;"),
    "input_grad_is_forward": (
        "d[si * W + sj] += f[a * K + b] * g[i * W + j];",
        "d[i * W + j] += f[a * K + b] * g[si * W + sj];"),
    "filter_grad_roles_swapped": (
        "sum += gp[i * W + j] * xp[si * W + sj];",
        "sum += gp[si * W + sj] * xp[i * W + j];"),
    "filter_grad_first_image_only": (
        "for (int64_t n = 0; n < N; ++n) {\n        const double* xp",
        "for (int64_t n = 0; n < 1; ++n) {\n        const double* xp"),
    "dense_taps_transposed": (
        "const double* f = w + ((o * K + a) * (int64_t)K + b) * Ci;\n            for (int64_t c = 0; c < Ci; ++c) sum",
        "const double* f = w + ((o * K + b) * (int64_t)K + a) * Ci;\n            for (int64_t c = 0; c < Ci; ++c) sum"),
    "upsample_coordinates_swapped": (
        "y[(pl * Ho + p) * Wo + q] = x[(pl * H + p / s) * W + q / s];",
        "y[(pl * Ho + p) * Wo + q] = x[(pl * H + q / s % H) * W + p / s % W];"),
    "upsample_rounds_to_nearest": (
        "y[(pl * Ho + p) * Wo + q] = x[(pl * H + p / s) * W + q / s];",
        "y[(pl * Ho + p) * Wo + q] = x[(pl * H + (p + s / 2) / s % H) * W + (q + s / 2) / s % W];"),
    "upsample_points_border_on_input": (
        "sum += f[a * K + b] * plane[(su / s) * W + sv / s];",
        "sum += f[a * K + b] * plane[(i / s + a - r < 0 ? 0 : su / s) * W + sv / s];"),
    "gray_weights_swapped": (
        "gray[n * P + p] = 0.299 * px[0] + 0.587 * px[P] + 0.114 * px[2 * P];",
        "gray[n * P + p] = 0.114 * px[0] + 0.587 * px[P] + 0.299 * px[2 * P];"),
    "dense_grad_sign": (
        "sum += dy[((n * H + i) * W + j) * Co + o] * x[((n * H + si) * W + sj) * Ci + c];",
        "sum -= dy[((n * H + i) * W + j) * Co + o] * x[((n * H + si) * W + sj) * Ci + c];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "giga_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
    with tempfile.TemporaryDirectory() as d:
        c_path = os.path.join(d, "mutant.c")
        so_path = os.path.join(d, "mutant.so")
        open(c_path, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                        "-std=c11", "-o", so_path, c_path], check=True)
        failed = []
        with oracle.use_library(so_path):
            for pin in PINS:
                try:
                    pin()
                except AssertionError:
                    failed.append(pin.__name__)
                    break
        assert failed, f"no pin catches the planted mistake {name}"
