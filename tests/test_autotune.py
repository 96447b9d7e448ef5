"""The depthwise autotuner's timing path on the GPU (giga_autotune_conv2d and
the on-demand tuning of mode 2): every op is benchmarked on a problem of
2 x 3 x 520 x 1000 (32 tiles of 64 x 128 per plane plus ragged tails), the
recorded choice is a valid candidate, the entry points then run with it and
match the FP64 oracle, and a saved cache reloads to the same choices."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from helpers import assert_fp32, poison_like, to_np

pytestmark = pytest.mark.gpu

SHAPE = (2, 3, 520, 1000)
# candidates per op: forward / input gradient 8, filter gradient 5, fused 7
OPS = {1: 8, 2: 8, 4: 5, 6: 7}


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


class _Mode:
    def __init__(self, mode):
        self.want = mode

    def __enter__(self):
        from paper_2504_01266_gb300 import _lib
        self.mode = _lib.giga_autotune_get_mode()
        _lib.giga_autotune_clear()
        _lib.giga_autotune_set_mode(self.want)

    def __exit__(self, *exc):
        from paper_2504_01266_gb300 import _lib
        _lib.giga_autotune_clear()
        _lib.giga_autotune_set_mode(self.mode)


def _data(K, seed):
    gen = torch.Generator().manual_seed(seed)
    x = torch.rand(SHAPE, generator=gen)
    w = torch.randn((SHAPE[1], K, K), generator=gen) * 0.1
    dy = torch.randn(SHAPE, generator=gen)
    return x, w, dy


@pytest.mark.parametrize("K,border", [(7, "clamp"), (3, "zero"), (15, "clamp")])
def test_tuner_records_valid_choices_that_the_entry_points_use(giga, tmp_path, K, border):
    from paper_2504_01266_gb300 import _lib as L
    b = {"zero": oracle.ZERO, "clamp": oracle.CLAMP}[border]
    x, w, dy = _data(K, 900 + K)
    xc, wc, dyc = x.cuda(), w.cuda(), dy.cuda()
    N, C, H, W = SHAPE
    d = L.desc(N, C, C, H, W, K, C, b, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)
    y, dx = torch.empty_like(xc), torch.empty_like(dyc)
    dw = torch.empty((C, K, K), device="cuda")
    wsb = L.giga_conv2d_workspace_size(d, L.GIGA_OP_BWD_INPUT | L.GIGA_OP_BWD_FILTER)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    with _Mode(2):
        for op in OPS:
            L.check(L.giga_autotune_conv2d(d, op, xc.data_ptr(), wc.data_ptr(), y.data_ptr(),
                                           dyc.data_ptr(), dx.data_ptr(), dw.data_ptr(),
                                           ws.data_ptr(), wsb, sp), f"autotune op {op}")
        choice = {op: L.giga_autotune_choice(d, op) for op in OPS}
        for op, n in OPS.items():
            assert 0 <= choice[op] < n, (op, choice[op])
        # the entry points run with the recorded choices
        y = giga.conv2d_fwd(xc, wc, border, out=poison_like(xc))
        dx_only = giga.conv2d_bwd_input(dyc, wc, border, out=poison_like(dyc))
        dw_only = giga.conv2d_bwd_filter(xc, dyc, K, border)
        dx, dw = giga.conv2d_bwd(xc, dyc, wc, border, dx=poison_like(dyc))
        torch.cuda.synchronize()
        xr, dyr, wn = x.double().numpy(), dy.double().numpy(), w.numpy()
        assert_fp32(to_np(y), oracle.dw_fwd(xr, wn, b), oracle.dw_fwd(np.abs(xr), np.abs(wn), b),
                    K * K, "fwd")
        ref_dx = oracle.dw_bwd_input(dyr, wn, b)
        mag_dx = oracle.dw_bwd_input(np.abs(dyr), np.abs(wn), b)
        for out in (dx_only, dx):
            assert_fp32(to_np(out), ref_dx, mag_dx, (K // 2 + 1) ** 2 * K * K, "dx")
        ref_dw = oracle.dw_bwd_filter(xr, dyr, K, b)
        mag_dw = oracle.dw_bwd_filter(np.abs(xr), np.abs(dyr), K, b)
        for out in (dw_only, dw):
            assert_fp32(to_np(out), ref_dw, mag_dw, N * H * W, "dw")
        # save, clear, load: the same choices come back
        path = str(tmp_path / "tuned.json")
        L.check(L.giga_autotune_save(path), "save")
        entries = json.load(open(path))["entries"]
        assert len(entries) == len(OPS)
        L.giga_autotune_clear()
        assert all(L.giga_autotune_choice(d, op) == 0 for op in OPS)
        L.check(L.giga_autotune_load(path), "load")
        assert {op: L.giga_autotune_choice(d, op) for op in OPS} == choice


def test_mode_full_tunes_an_uncached_problem_on_first_use(giga, tmp_path):
    """In mode 2 the first call for an uncached problem class benchmarks its
    candidates (outside any capture) and records the choice."""
    from paper_2504_01266_gb300 import _lib as L
    K = 5
    x, w, dy = _data(K, 950)
    xc, wc = x.cuda(), w.cuda()
    with _Mode(2):
        path = str(tmp_path / "empty.json")
        L.check(L.giga_autotune_save(path), "save")
        assert json.load(open(path))["entries"] == {}
        y = giga.conv2d_fwd(xc, wc, "zero", out=poison_like(xc))
        torch.cuda.synchronize()
        L.check(L.giga_autotune_save(path), "save")
        entries = json.load(open(path))["entries"]
        assert len(entries) == 1 and 0 <= list(entries.values())[0] < 8
        xr, wn = x.double().numpy(), w.numpy()
        assert_fp32(to_np(y), oracle.dw_fwd(xr, wn, oracle.ZERO),
                    oracle.dw_fwd(np.abs(xr), np.abs(wn), oracle.ZERO), K * K, "fwd")


def test_giga_log_prints_tuning_decisions(giga, capfd):
    """GIGA_LOG=1: every tuning decision is printed to standard error with
    the time of each candidate."""
    from paper_2504_01266_gb300 import _lib as L
    x, w, dy = _data(3, 960)
    xc, wc = x.cuda(), w.cuda()
    N, C, H, W = SHAPE
    d = L.desc(N, C, C, H, W, 3, C, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)
    y = torch.empty_like(xc)
    old = os.environ.get("GIGA_LOG")
    os.environ["GIGA_LOG"] = "1"
    try:
        with _Mode(1):
            capfd.readouterr()
            L.check(L.giga_autotune_conv2d(d, 1, xc.data_ptr(), wc.data_ptr(), y.data_ptr(),
                                           0, 0, 0, 0, 0, torch.cuda.current_stream().cuda_stream),
                    "autotune")
            err = capfd.readouterr().err
    finally:
        if old is None:
            del os.environ["GIGA_LOG"]
        else:
            os.environ["GIGA_LOG"] = old
    line = [ln for ln in err.splitlines() if ln.startswith("giga autotune: forward f32 K=3 zero")]
    assert len(line) == 1, err
    assert "candidate" in line[0] and line[0].count(":") >= 8 + 1
