"""Ragged batches in one persistent launch: parity with the per-image path and
with the FP64 oracle, CUDA-graph replay, determinism, and the argument checks
of the plan API."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import FP32_TOL, assert_fp32, normwise, to_np

ALL = 7  # GIGA_OP_FWD | GIGA_OP_BWD_INPUT | GIGA_OP_BWD_FILTER


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def batch(imgs, dev="cuda"):
    out = []
    for im in imgs:
        x, dy = im.x[0].to(dev), im.dy[0].to(dev)
        out.append({"x": x, "dy": dy, "w": im.w.to(dev),
                    "y": torch.full_like(x, float("nan")), "dx": torch.full_like(dy, float("nan")),
                    "dw": torch.full((x.shape[0], im.K, im.K), float("nan"), device=dev)})
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_ragged_matches_oracle(giga, border):
    imgs = workloads.ragged(n=12, lo=5, hi=300, ks=(1, 3, 5, 7, 9, 11, 13, 15))
    b = batch(imgs)
    plan = giga.BatchedPlan(b, ALL, border)
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    bo = oracle.ZERO if border == "zero" else oracle.CLAMP
    for im, t in zip(imgs, b):
        x, w, dy, K = im.x.numpy(), im.w.numpy(), im.dy.numpy(), im.K
        ax, aw, ady = np.abs(x), np.abs(w), np.abs(dy)
        assert_fp32(to_np(t["y"])[None], oracle.dw_fwd(x, w, bo), oracle.dw_fwd(ax, aw, bo),
                    K * K, ("y", im.H, im.W, K))
        assert_fp32(to_np(t["dx"])[None], oracle.dw_bwd_input(dy, w, bo),
                    oracle.dw_bwd_input(ady, aw, bo), (K // 2 + 1) ** 2 * K * K,
                    ("dx", im.H, im.W, K))
        assert_fp32(to_np(t["dw"]), oracle.dw_bwd_filter(x, dy, K, bo),
                    oracle.dw_bwd_filter(ax, ady, K, bo), im.H * im.W, ("dw", im.H, im.W, K))
    plan.close()


@pytest.mark.gpu
def test_ragged_equals_per_image_path_and_graph_replay(giga):
    imgs = workloads.ragged(n=20, lo=64, hi=700)
    b = batch(imgs)
    plan = giga.BatchedPlan(b, ALL, "zero")
    plan.upload()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
    for t in b:
        for k in ("y", "dx", "dw"):
            t[k].fill_(float("nan"))
    graph.replay()
    graph.replay()  # twice: counters are reset inside the graph
    torch.cuda.synchronize()
    for im, t in zip(imgs, b):
        x, dy, w = im.x.cuda(), im.dy.cuda(), im.w.cuda()
        y = giga.conv2d_fwd(x, w, "zero")
        dx, dw = giga.conv2d_bwd(x, dy, w, "zero")
        # same arithmetic order per pixel -> identical forward and input gradient
        assert torch.equal(t["y"], y[0]), (im.H, im.W, im.K)
        assert torch.equal(t["dx"], dx[0]), (im.H, im.W, im.K)
        assert normwise(to_np(t["dw"]), to_np(dw)) <= FP32_TOL
    plan.close()


@pytest.mark.gpu
def test_ragged_subsets_of_ops_and_determinism(giga):
    imgs = workloads.ragged(n=6, lo=30, hi=260, ks=(3, 11))
    b = batch(imgs)
    p1 = giga.BatchedPlan([{"x": t["x"], "dy": t["dy"], "dw": t["dw"]} for t in b], 4, "clamp")
    p1.upload(); p1.run()
    first = [t["dw"].clone() for t in b]
    p1.run()
    torch.cuda.synchronize()
    for f, t in zip(first, b):
        assert torch.equal(f, t["dw"])
    p2 = giga.BatchedPlan([{"dy": t["dy"], "w": t["w"], "dx": t["dx"]} for t in b], 2, "clamp")
    p2.upload(); p2.run()
    torch.cuda.synchronize()
    for im, t in zip(imgs, b):
        ref = oracle.dw_bwd_input(im.dy.numpy(), im.w.numpy(), oracle.CLAMP)
        assert normwise(to_np(t["dx"])[None], ref) <= FP32_TOL
    p1.close(); p2.close()


@pytest.mark.gpu
def test_ragged_bf16(giga):
    imgs = workloads.ragged(n=5, lo=40, hi=300, ks=(3, 9), dtype=torch.bfloat16)
    b = batch(imgs)
    plan = giga.BatchedPlan(b, ALL, "zero", dtype=torch.bfloat16)
    plan.upload(); plan.run()
    torch.cuda.synchronize()
    for im, t in zip(imgs, b):
        xr, dyr = im.x.float().numpy(), im.dy.float().numpy()
        assert normwise(to_np(t["y"])[None], oracle.dw_fwd(xr, im.w.numpy(), 0)) <= 2 ** -8
        assert normwise(to_np(t["dx"])[None], oracle.dw_bwd_input(dyr, im.w.numpy(), 0)) <= 2 ** -8
        assert normwise(to_np(t["dw"]), oracle.dw_bwd_filter(xr, dyr, im.K, 0)) <= FP32_TOL
    plan.close()


@pytest.mark.gpu
def test_ragged_autotune_chunk_sizes(giga):
    """The plan's autotuner times 1 to 32 tiles per chunk (powers of 2), keeps one;
    every chunk size gives the same y and dx bit for bit (per-pixel arithmetic
    does not depend on the chunking) and a filter gradient within the FP32
    bound; the tuned plan captures and replays in a CUDA graph; the tuner
    refuses to run while the stream is capturing."""
    imgs = workloads.ragged(n=10, lo=40, hi=600, ks=(3, 5, 9, 11))
    b = batch(imgs)
    plan = giga.BatchedPlan(b, ALL, "zero")
    assert plan.tiles_per_chunk == 4
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    ref = [(t["y"].clone(), t["dx"].clone(), t["dw"].clone()) for t in b]
    tpc = plan.autotune()
    assert tpc in (1, 2, 4, 8, 16, 32) and plan.tiles_per_chunk == tpc
    for t in b:
        for k in ("y", "dx", "dw"):
            t[k].fill_(float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
            from paper_2504_01266_gb300 import _lib
            with pytest.raises(_lib.GigaError):
                plan.autotune()
    graph.replay()
    torch.cuda.synchronize()
    for im, t, (y, dx, dw) in zip(imgs, b, ref):
        assert torch.equal(t["y"], y) and torch.equal(t["dx"], dx)
        x, dyn = im.x.numpy(), im.dy.numpy()
        assert_fp32(to_np(t["dw"]), oracle.dw_bwd_filter(x, dyn, im.K, 0),
                    oracle.dw_bwd_filter(np.abs(x), np.abs(dyn), im.K, 0), im.H * im.W,
                    ("dw", im.H, im.W, im.K, tpc))
    plan.close()


@pytest.mark.gpu
def test_run_requires_the_uploaded_workspace(giga):
    """The kernels index the tile table in the workspace: a run with another
    workspace than the one the table went to is refused before any launch."""
    from paper_2504_01266_gb300 import _lib
    imgs = workloads.ragged(n=3, lo=20, hi=90, ks=(3, 5))
    b = batch(imgs)
    plan = giga.BatchedPlan(b, ALL, "zero")
    with pytest.raises(_lib.GigaError):
        plan.run()                                   # never uploaded
    plan.upload()
    other = torch.empty_like(plan.ws)
    st = _lib.giga_batched_plan_run(plan.plan, other.data_ptr(), other.numel(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == _lib.GIGA_ERR_WORKSPACE
    plan.run()
    torch.cuda.synchronize()
    for im, t in zip(imgs, b):
        y = giga.conv2d_fwd(im.x.cuda(), im.w.cuda(), "zero")
        assert torch.equal(t["y"], y[0])
    plan.close()


@pytest.mark.gpu
def test_ragged_workload_sampled(giga):
    """The benchmark's ragged batch (256 three-channel images, sides 64-4096,
    K in {3, 5, 9, 11}, zero border, inputs drawn on the device as the
    benchmark draws them) in one autotuned persistent launch: every output is
    written, and every 16th image is checked on sampled y and dx pixels (every
    kind of border pixel included) and on filter-gradient taps."""
    shapes = workloads.ragged_shapes()
    imgs = []
    for i, (h, w_, k) in enumerate(shapes):
        g = workloads.generator("ragged", salt=i + 1, device="cuda")
        x = torch.rand((3, h, w_), generator=g, device="cuda")
        wt = torch.randn((3, k, k), generator=g, device="cuda") * 0.1
        dy = torch.randn((3, h, w_), generator=g, device="cuda")
        imgs.append({"x": x, "dy": dy, "w": wt, "y": torch.full_like(x, float("nan")),
                     "dx": torch.full_like(x, float("nan")),
                     "dw": torch.full((3, k, k), float("nan"), device="cuda")})
    plan = giga.BatchedPlan(imgs, ALL, "zero")
    plan.upload()
    plan.autotune()
    for t in imgs:
        for key in ("y", "dx", "dw"):
            t[key].fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    assert not any(torch.isnan(t[key]).any().item() for t in imgs for key in ("y", "dx", "dw"))
    for i in range(0, len(shapes), 16):
        h, w_, k = shapes[i]
        t = imgs[i]
        x, dyn, wn = t["x"].cpu()[None].numpy(), t["dy"].cpu()[None].numpy(), t["w"].cpu().numpy()
        idx = torch.unique(torch.cat([workloads.sample_indices(x.size, 300, salt=i),
                                      workloads.border_indices(1, 3, h, w_, 1, salt=i)]))
        ii = idx.numpy()
        got_y = t["y"].reshape(-1)[idx.cuda()].double().cpu().numpy()
        got_dx = t["dx"].reshape(-1)[idx.cuda()].double().cpu().numpy()
        assert normwise(got_y, oracle.dw_fwd_points(x, wn, oracle.ZERO, ii)) <= FP32_TOL, i
        assert normwise(got_dx, oracle.dw_bwd_input_points(dyn, wn, oracle.ZERO, ii)) <= FP32_TOL, i
        taps = np.array([0, k * k // 2, k * k + 1, 3 * k * k - 1])
        ref_dw = oracle.dw_bwd_filter_taps(x, dyn, k, oracle.ZERO, taps)
        got_dw = to_np(t["dw"]).reshape(-1)[taps]
        assert np.abs(got_dw - ref_dw).max() <= FP32_TOL * np.abs(ref_dw).max(), i
    plan.close()


# ------------------------------------------------------- host-side checks

def _img(lib, H=10, W=10, C=1, K=3, p=0x100000):
    return lib.giga_image_t(p, p * 2, p * 3, p * 4, p * 5, p * 6, H, W, C, K)


def test_plan_rejects_bad_arguments():
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    arr = (_lib.giga_image_t * 1)(_img(_lib, K=4))
    with pytest.raises(_lib.GigaError):
        _lib.giga_batched_plan_create(arr, 1, ALL, 0, 0)
    arr = (_lib.giga_image_t * 1)(_img(_lib, K=17))
    with pytest.raises(_lib.GigaError) as e:
        _lib.giga_batched_plan_create(arr, 1, ALL, 0, 0)
    assert e.value.status == _lib.GIGA_ERR_UNSUPPORTED
    arr = (_lib.giga_image_t * 1)(_img(_lib))
    with pytest.raises(_lib.GigaError):
        _lib.giga_batched_plan_create(arr, 1, 0, 0, 0)        # no ops
    bad = _img(_lib)
    bad.x = 0x100001                                          # misaligned
    arr = (_lib.giga_image_t * 1)(bad)
    with pytest.raises(_lib.GigaError) as e:
        _lib.giga_batched_plan_create(arr, 1, ALL, 0, 0)
    assert e.value.status == _lib.GIGA_ERR_MISALIGNED


def test_plan_workspace_size_covers_table_and_partials():
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    arr = (_lib.giga_image_t * 2)(_img(_lib, H=100, W=300, C=3, K=5),
                                  _img(_lib, H=64, W=128, C=3, K=15))
    n = _lib.giga_conv2d_batched_workspace_size(arr, 2, ALL)
    tiles0 = ((300 + 127) // 128) * ((100 + 63) // 64)       # 6 tiles -> 2 chunks per channel
    partial_floats = 3 * 2 * 25 + 3 * 1 * 225
    assert n >= partial_floats * 4 + (3 * 2 + 3) * 16 and n % 256 == 0
    assert tiles0 == 6


def test_plan_workspace_covers_every_chunk_size_and_autotune_argument_checks():
    """The plan's workspace is sized for the smallest chunks (one tile each),
    so the autotuner can switch chunk sizes inside it; the tuner's argument
    checks run before any CUDA call."""
    from paper_2504_01266_gb300 import _lib, build
    build.build()
    arr = (_lib.giga_image_t * 2)(_img(_lib, H=100, W=300, C=3, K=5),
                                  _img(_lib, H=64, W=128, C=3, K=15))
    n = _lib.giga_conv2d_batched_workspace_size(arr, 2, ALL)
    # one tile per chunk: 6 chunks per channel for image 0, 1 for image 1
    partial_floats = 3 * 6 * 25 + 3 * 1 * 225
    chunks = 3 * 6 + 3 * 1
    assert n >= partial_floats * 4 + chunks * 16 and n % 256 == 0
    plan = _lib.giga_batched_plan_create(arr, 2, ALL, 0, 0)
    assert _lib.giga_batched_plan_workspace_size(plan) == n
    assert _lib.giga_batched_plan_tiles_per_chunk(plan) == 4
    lib = _lib.load()
    assert lib.giga_batched_plan_autotune(None, 0x10000, n, None, None) == \
        _lib.GIGA_ERR_INVALID_ARG
    assert lib.giga_batched_plan_autotune(plan, None, n, None, None) == _lib.GIGA_ERR_WORKSPACE
    assert lib.giga_batched_plan_autotune(plan, 0x10000, n - 1, None, None) == \
        _lib.GIGA_ERR_WORKSPACE
    assert lib.giga_batched_plan_autotune(plan, 0x10010, n, None, None) == \
        _lib.GIGA_ERR_WORKSPACE
    # never uploaded: run refuses before any launch
    assert _lib.giga_batched_plan_run(plan, 0x10000, n, None) == _lib.GIGA_ERR_INVALID_ARG
    assert _lib.giga_batched_plan_tiles_per_chunk(None) == -1
    _lib.giga_batched_plan_destroy(plan)
