"""The sharpening benchmark over a ragged batch of images (upsample by a
per-image scale, then a per-image depthwise filter; Sections 5 and 6.6) in one
persistent launch: parity with the FP64 oracle image by image, equality with
the single-image fused pass, CUDA-graph replay, the full database on sampled
outputs, and the plan's argument checks (host only, no GPU needed)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import BF16_KERNEL_TOL, assert_fp32, normwise, to_np
from paper_2504_01266_gb300 import _lib

BORDER = {"zero": oracle.ZERO, "clamp": oracle.CLAMP}


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def small_batch(n, seed, dtype=torch.float32, ks=(1, 3, 5, 7, 9, 11, 13, 15)):
    """n images of 1-3 channels, sides 1-70, scales 2-9, every supported K;
    several output tiles per image and ragged tails in both directions."""
    g = torch.Generator().manual_seed(seed)
    out = []
    for i in range(n):
        C = int(torch.randint(1, 4, (1,), generator=g))
        H = int(torch.randint(1, 71, (1,), generator=g))
        W = int(torch.randint(1, 71, (1,), generator=g))
        s = int(torch.randint(2, 10, (1,), generator=g))
        K = ks[i % len(ks)]
        x = torch.rand((C, H, W), generator=g).to(dtype)
        w = torch.randn((C, K, K), generator=g) * 0.1
        out.append({"x": x, "w": w, "scale": s})
    return out


def to_device(imgs, dtype):
    dev = []
    for im in imgs:
        C, H, W = im["x"].shape
        s = im["scale"]
        dev.append({"x": im["x"].cuda(), "w": im["w"].cuda(), "scale": s,
                    "y": torch.full((C, H * s, W * s), float("nan"), dtype=dtype,
                                    device="cuda")})
    return dev


@pytest.mark.gpu
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_batched_fp32_matches_oracle_and_single_image_path(giga, border):
    imgs = small_batch(16, 31 + len(border))
    dev = to_device(imgs, torch.float32)
    plan = giga.UpsampleBatchedPlan(dev, border)
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    b = BORDER[border]
    for im, d in zip(imgs, dev):
        x, w, s = im["x"].numpy()[None], im["w"].numpy(), im["scale"]
        K = w.shape[-1]
        ref = oracle.upsample_dw_fwd(x, w, b, s)
        mag = oracle.upsample_dw_fwd(np.abs(x), np.abs(w), b, s)
        assert_fp32(to_np(d["y"])[None], ref, mag, K * K, (x.shape, s, K, border))
        single = giga.upsample_conv2d(d["x"][None], d["w"], s, border)
        assert torch.equal(d["y"], single[0]), (x.shape, s, K, border)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("border", ["zero", "clamp"])
def test_batched_bf16_matches_oracle(giga, border):
    imgs = small_batch(10, 77, torch.bfloat16, ks=(3, 5, 9, 11, 15))
    dev = to_device(imgs, torch.bfloat16)
    plan = giga.UpsampleBatchedPlan(dev, border, torch.bfloat16)
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    for im, d in zip(imgs, dev):
        x, w, s = im["x"].double().numpy()[None], im["w"].numpy(), im["scale"]
        ref = oracle.upsample_dw_fwd(x, w, BORDER[border], s)
        got = to_np(d["y"])[None]
        assert not np.isnan(got).any()
        assert normwise(got, ref) <= BF16_KERNEL_TOL, (x.shape, s, w.shape, border)
        single = giga.upsample_conv2d(d["x"][None], d["w"], s, border)
        assert torch.equal(d["y"], single[0])
    plan.close()


@pytest.mark.gpu
def test_graph_replay_and_repeated_runs(giga):
    imgs = small_batch(24, 5)
    dev = to_device(imgs, torch.float32)
    plan = giga.UpsampleBatchedPlan(dev, "zero")
    plan.upload()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
    torch.cuda.synchronize()
    for d in dev:
        d["y"].fill_(float("nan"))
    graph.replay()
    graph.replay()  # the work counter is reset inside the graph
    torch.cuda.synchronize()
    first = [d["y"].clone() for d in dev]
    for d in dev:
        d["y"].fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    for a, d in zip(first, dev):
        single = giga.upsample_conv2d(d["x"][None], d["w"], d["scale"], "zero")[0]
        assert torch.equal(a, single) and torch.equal(d["y"], single)
    plan.close()


@pytest.mark.gpu
def test_empty_images_and_empty_batch(giga):
    imgs = small_batch(3, 9)
    dev = to_device(imgs, torch.float32)
    zero = {"x": torch.empty((3, 0, 5), device="cuda"), "w": torch.zeros((3, 3, 3), device="cuda"),
            "scale": 4, "y": torch.empty((3, 0, 20), device="cuda")}
    plan = giga.UpsampleBatchedPlan(dev[:1] + [zero] + dev[1:], "clamp")
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    for d in dev:
        single = giga.upsample_conv2d(d["x"][None], d["w"], d["scale"], "clamp")[0]
        assert torch.equal(d["y"], single)
    plan.close()
    empty = giga.UpsampleBatchedPlan([], "zero")
    empty.upload()
    empty.run()
    empty.close()


@pytest.mark.gpu
def test_run_requires_the_uploaded_workspace(giga):
    imgs = small_batch(2, 13)
    dev = to_device(imgs, torch.float32)
    plan = giga.UpsampleBatchedPlan(dev, "zero")
    with pytest.raises(_lib.GigaError):
        plan.run()                                   # never uploaded
    plan.upload()
    other = torch.empty_like(plan.ws)
    st = _lib.giga_upsample_batched_plan_run(plan.plan, other.data_ptr(), other.numel(),
                                             torch.cuda.current_stream().cuda_stream)
    assert st == _lib.GIGA_ERR_WORKSPACE
    plan.run()
    torch.cuda.synchronize()
    for d in dev:
        single = giga.upsample_conv2d(d["x"][None], d["w"], d["scale"], "zero")[0]
        assert torch.equal(d["y"], single)
    plan.close()


@pytest.mark.gpu
def test_database_workload_sampled(giga):
    """The benchmark's database (128 images, sides 64-1024, scales 2-8,
    K in {3, 5, 9, 11}, zero border) in one launch: sampled outputs and every
    kind of border pixel of each image against the oracle."""
    shapes = workloads.up_ragged_shapes()
    imgs, dev = [], []
    for i, (H, W, s, K) in enumerate(shapes):
        x, w = workloads.up_ragged_image(i, H, W, K)
        imgs.append((x, w, s))
        dev.append({"x": x.cuda(), "w": w.cuda(), "scale": s,
                    "y": torch.full((3, H * s, W * s), float("nan"), device="cuda")})
    plan = giga.UpsampleBatchedPlan(dev, "zero")
    plan.upload()
    plan.run()
    torch.cuda.synchronize()
    worst = 0.0
    for i, ((x, w, s), d) in enumerate(zip(imgs, dev)):
        C, Ho, Wo = d["y"].shape
        idx = torch.unique(torch.cat([workloads.sample_indices(d["y"].numel(), 200, salt=i),
                                      workloads.border_indices(1, C, Ho, Wo, 1, salt=i)]))
        got = d["y"].reshape(-1)[idx.cuda()].double().cpu().numpy()
        ref = oracle.upsample_dw_fwd_points(x.numpy()[None], w.numpy(), oracle.ZERO, s,
                                            idx.numpy())
        mag = oracle.upsample_dw_fwd_points(np.abs(x.numpy()[None]), np.abs(w.numpy()),
                                            oracle.ZERO, s, idx.numpy())
        K = w.shape[-1]
        assert_fp32(got, ref, mag, K * K, ("image", i, s, K))
        worst = max(worst, normwise(got, ref))
        assert not torch.isnan(d["y"]).any(), ("unwritten output", i)
    plan.close()
    assert worst <= 1e-5


# ------------------------------------------------------------ host-only checks

def up_images(specs):
    arr = (_lib.giga_up_image_t * max(1, len(specs)))()
    for i, (H, W, C, K, s, x, y, w) in enumerate(specs):
        arr[i] = _lib.giga_up_image_t(x, y, w, H, W, C, K, s, 0)
    return arr


A, B, Wt = 0x100000, 0x40000000, 0x20000


@pytest.fixture(scope="module")
def lib():
    from paper_2504_01266_gb300 import build
    build.build()
    return _lib.load()


@pytest.mark.parametrize("spec,status", [
    ((8, 8, 3, 3, 1, A, B, Wt), _lib.GIGA_ERR_UNSUPPORTED),     # scale 1: the plain filter
    ((8, 8, 3, 3, 0, A, B, Wt), _lib.GIGA_ERR_INVALID_ARG),     # scale 0
    ((8, 8, 3, 17, 2, A, B, Wt), _lib.GIGA_ERR_UNSUPPORTED),    # K above 15
    ((8, 8, 3, 4, 2, A, B, Wt), _lib.GIGA_ERR_INVALID_ARG),     # even K
    ((8, -1, 3, 3, 2, A, B, Wt), _lib.GIGA_ERR_INVALID_ARG),    # negative side
    ((8, 8, 3, 3, 2, None, B, Wt), _lib.GIGA_ERR_INVALID_ARG),  # NULL x
    ((8, 8, 3, 3, 2, A + 2, B, Wt), _lib.GIGA_ERR_MISALIGNED),  # misaligned x
    ((8, 8, 3, 3, 2, A, A + 64, Wt), _lib.GIGA_ERR_INVALID_ARG),  # y overlaps x
    ((1 << 20, 8, 3, 3, 4096, A, B, Wt), _lib.GIGA_ERR_INVALID_ARG),  # side of 2^32
])
def test_plan_rejects_bad_images(lib, spec, status):
    arr = up_images([(16, 16, 3, 5, 3, A, B, Wt), spec])
    import ctypes
    plan = _lib._P(None)
    got = lib.giga_upsample_batched_plan_create(arr, 2, _lib.GIGA_BORDER_ZERO, _lib.GIGA_F32,
                                                ctypes.byref(plan))
    assert got == status, _lib.last_error_detail()
    assert not plan.value
    assert "image 1" in _lib.last_error_detail()


def test_plan_workspace_and_reserved(lib):
    import ctypes
    arr = up_images([(16, 16, 3, 5, 3, A, B, Wt), (40, 7, 1, 15, 9, A, B, Wt)])
    n = _lib.giga_upsample_conv2d_batched_workspace_size(arr, 2)
    assert n >= 2 * 64 and n % 256 == 0
    plan = _lib.giga_upsample_batched_plan_create(arr, 2, _lib.GIGA_BORDER_CLAMP, _lib.GIGA_BF16)
    assert _lib.giga_upsample_batched_plan_workspace_size(plan) == n
    # the workspace is checked before any CUDA call
    assert _lib.giga_upsample_batched_plan_run(plan, None, 0, None) == _lib.GIGA_ERR_WORKSPACE
    assert _lib.giga_upsample_batched_plan_upload(plan, 0x10010, n, None) == \
        _lib.GIGA_ERR_WORKSPACE
    assert _lib.giga_upsample_batched_plan_run(plan, 0x10000, n - 1, None) == \
        _lib.GIGA_ERR_WORKSPACE
    _lib.giga_upsample_batched_plan_destroy(plan)
    arr[0].reserved = 1
    p = _lib._P(None)
    assert lib.giga_upsample_batched_plan_create(arr, 2, 0, 0, ctypes.byref(p)) == \
        _lib.GIGA_ERR_INVALID_ARG
    assert "reserved" in _lib.last_error_detail()
    arr[0].reserved = 0
    assert lib.giga_upsample_batched_plan_create(arr, 2, 7, 0, ctypes.byref(p)) == \
        _lib.GIGA_ERR_INVALID_ARG
    assert "border" in _lib.last_error_detail()
