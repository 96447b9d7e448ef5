"""Benchmark of the depthwise filtering hot path (forward + both gradients).

Workload (per GPU): 8 x 3 x 4096 x 4096 FP32 images, pixels uniform [0, 1),
depthwise K x K filters normal(0, 0.1) for K in {3, 7, 15}, clamp border,
upstream gradient normal(0, 1).  One step = for every K: the forward filter
and the fused backward pass (input gradient + filter gradient), all through
the C ABI.  Metric: Gpixel*tap/s = sum_K 3 * N*C*H*W*K^2 / step time.

Prints ONE JSON line.  `--impl reference` times the FP64 CPU oracle (there
is no other reference implementation of this path) on a bounded sample of
the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the
data path; value = work of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, C, H, W = 8, 3, 4096, 4096
KS = (3, 7, 15)
# DRAM bytes (read + written) per pixel of one launch, from the ncu capture of
# one 1x3x4096x4096 launch of the kernel (dram__bytes_read.sum 201.416 MB +
# dram__bytes_write.sum 153.949 MB); traffic grows with the pixel count, so a
# launch over 8 such images moves 8x that.
NCU_DRAM_BYTES_PER_PX = {
    "dw_fwd_kernel<float,15,8>": (201415680 + 153949184) / (3 * 4096 * 4096),
}
METRIC = "Gpixel*tap/s fwd+bwd (depthwise KxK, K in {3,7,15})"
UNIT = "Gpixel*tap/s"
WORKLOAD = "plain_scale: 8x3x4096x4096 fp32, depthwise K in {3,7,15} normal(0,0.1), clamp border, fwd+bwd"
FP32_LANES, SM_MAX_MHZ = 128, 2070.0   # FP32 FMA lanes per SM; fallback max SM clock
RAGGED_IMAGES = None   # all 256 images of the ragged workload; a prefix for profiling runs
# FP32 FMA throughput measured on this device by the library's own kernel
# (giga_fp32_fma_peak) and the device's SM count; set by measure_fp32_peak()
FP32_MEASURED = {}


def peaks():
    """Roofline denominators: HBM from MEASURED_PEAKS.json (the driver's copy
    benchmark), FP32 FMA from this run's measurement when it has been taken,
    else derived from the SM count, lanes and maximum clock."""
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "source": "measured"}
        mhz = float(m.get("sm_max_mhz", SM_MAX_MHZ))
    except Exception:
        mhz = SM_MAX_MHZ
    sms = FP32_MEASURED.get("sms", 152)
    p["sms"] = sms
    p["fp32_tflops_derived"] = sms * FP32_LANES * 2 * mhz * 1e6 / 1e12
    if FP32_MEASURED.get("tflops"):
        p["fp32_tflops"] = FP32_MEASURED["tflops"]
        p["fp32_source"] = (f"measured: giga_fp32_fma_peak (16 FMA chains/thread, {sms} SMs, "
                            f"best of plain and packed f32x2)")
    else:
        p["fp32_tflops"] = p["fp32_tflops_derived"]
        p["fp32_source"] = f"derived: {sms} SMs x {FP32_LANES} lanes x 2 x {mhz:.0f} MHz"
    return p


def measure_fp32_peak(dev):
    """FP32 FMA throughput of this GPU (plain and packed FMA) and its SM count."""
    import torch
    from paper_2504_01266_gb300 import _lib as L
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nb = L.giga_fp32_fma_peak_sink_bytes()
    sink = torch.empty(nb, dtype=torch.uint8, device=dev)
    sp = torch.cuda.current_stream(dev).cuda_stream
    plain, _ = L.giga_fp32_fma_peak(0, sink.data_ptr(), nb, sp)
    packed, _ = L.giga_fp32_fma_peak(1, sink.data_ptr(), nb, sp)
    FP32_MEASURED.update({"sms": sms, "plain": plain, "packed": packed,
                          "tflops": max(plain, packed)})
    return FP32_MEASURED


def _r(v, digits=4):
    """Round floats (recursively) to `digits` significant digits for the line."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}")
    if isinstance(v, dict):
        return {k: _r(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_r(x, digits) for x in v]
    return v


def set_images(n: int):
    global N, WORKLOAD
    N = n
    WORKLOAD = WORKLOAD.replace("8x3x4096x4096", f"{n}x3x4096x4096")


def set_ragged_images(n: int):
    global RAGGED_IMAGES
    RAGGED_IMAGES = n


def taps_per_step():
    return sum(3 * N * C * H * W * K * K for K in KS)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, start: float, end: float):
        """Restrict the summary to samples taken in [start, end] (host time)."""
        self.window = (start, end)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = getattr(self, "window", (0.0, float("inf")))
        # a sample printed up to one period after the window still describes it
        lines = [ln for t, ln in self.lines if lo <= t <= hi + 0.05]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm), "period_ms": 50}


# ------------------------------------------------------------- distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank timing over all ranks (NCCL on GPU, gloo on CPU)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(work_per_rank: float, ms_local: float, world: int):
    """Whole-job throughput of independent replicas: the work of all ranks over
    the slowest rank's time.  Returns (value per second, max ms)."""
    ms = max_over_ranks(ms_local, world)
    return world * work_per_rank / (ms * 1e-3), ms


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------- CPU oracle

def oracle_sample_rate(rows: int = H, images: int = 1):
    """Time the FP64 oracle (fwd + input grad + filter grad for every K) on
    `rows` x 4096 pixels of one image's 3 channels (default: one whole image
    of the 8); returns (Gpixel*tap/s, threads, seconds, description)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(2504)
    x = rng.random((images, C, rows, W))
    dy = rng.standard_normal((images, C, rows, W))
    taps = 0
    t0 = time.perf_counter()
    for K in KS:
        w = rng.normal(0.0, 0.1, (C, K, K))
        oracle.dw_fwd(x, w, oracle.CLAMP)
        oracle.dw_bwd_input(dy, w, oracle.CLAMP)
        oracle.dw_bwd_filter(x, dy, K, oracle.CLAMP)
        taps += 3 * images * C * rows * W * K * K
    dt = time.perf_counter() - t0
    desc = (f"{images}x{C}x{rows}x{W} of the {N}x{C}x{H}x{W} workload, "
            f"fwd+bwd_input+bwd_filter for K in {list(KS)}, FP64")
    return taps / dt / 1e9, oracle.num_threads(), dt, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    rate_rows = 256
    times = []
    for step in range(args.warmup + args.steps):
        v, cores, dt, desc = oracle_sample_rate(rate_rows)
        if step >= args.warmup:
            times.append((v, dt))
    value = statistics.median(v for v, _ in times)
    ms = statistics.median(dt for _, dt in times) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# -------------------------------------------------------- comparisons

def _events(stream, fn, iters):
    """Median per-iteration milliseconds of fn() over `iters` runs, CUDA events
    on the launching stream, after one warm-up."""
    import torch
    fn()
    times = []
    for _ in range(iters):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def _normwise(got, ref):
    import numpy as np
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def compare_bf16(dev, iters, images=32, tune=True):
    """BF16 storage (FP32 accumulation) vs FP32 storage on 32 x 3 x 2048 x 2048,
    9 x 9 filters, zero border: fwd + fused bwd, with the normwise error of
    sampled outputs against the FP64 oracle (i) on the BF16-rounded inputs and
    (ii) on the FP32 originals.  `images` shrinks the batch for profiling runs;
    tune=False keeps the built-in default configurations (a fixed launch
    sequence for ncu)."""
    import torch
    import oracle
    import workloads
    from paper_2504_01266_gb300 import _lib as L
    Nb, Cb, Hb, Wb, Kb = images, 3, 2048, 2048, 9
    g = torch.Generator(device=dev)
    g.manual_seed(2504 + 4)
    x32 = torch.rand((Nb, Cb, Hb, Wb), generator=g, device=dev)
    dy32 = torch.randn((Nb, Cb, Hb, Wb), generator=g, device=dev)
    w = (torch.randn((Cb, Kb, Kb), generator=torch.Generator().manual_seed(2508)) * 0.1).to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    out = {}
    res = {}
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        x, dy = x32.to(dt), dy32.to(dt)
        y, dx = torch.empty_like(x), torch.empty_like(x)
        dw = torch.empty((Cb, Kb, Kb), device=dev)
        d = L.desc(Nb, Cb, Cb, Hb, Wb, Kb, Cb, 0, L.GIGA_F32 if dt == torch.float32 else L.GIGA_BF16,
                   L.GIGA_LAYOUT_NCHW)
        wsb = L.giga_conv2d_workspace_size(d, 6)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        if tune:
            L.check(L.giga_autotune_conv2d(d, 7, x.data_ptr(), w.data_ptr(), y.data_ptr(),
                                           dy.data_ptr(), dx.data_ptr(), dw.data_ptr(),
                                           ws.data_ptr(), wsb, sp), "autotune")

        def run():
            L.check(L.giga_conv2d_fwd(d, x.data_ptr(), w.data_ptr(), y.data_ptr(), None, 0, sp), "fwd")
            L.check(L.giga_conv2d_bwd(d, x.data_ptr(), dy.data_ptr(), w.data_ptr(), dx.data_ptr(),
                                      dw.data_ptr(), ws.data_ptr(), wsb, sp), "bwd")
        ms = _events(stream, run, iters)
        px = Nb * Cb * Hb * Wb
        out[name] = {"ms": ms, "value": 3 * px * Kb * Kb / (ms * 1e-3) / 1e9,
                     "bytes_per_px": (20 if dt == torch.float32 else 10)}
        res[name] = (x, dy, y, dx, dw)
        del ws
    # sampled errors against the FP64 oracle (one image's planes, 1500 points)
    idx = workloads.sample_indices(Cb * Hb * Wb, 1500, salt=9)
    xb0 = res["bf16"][0][0:1].float().cpu().numpy()
    dyb0 = res["bf16"][1][0:1].float().cpu().numpy()
    x0, dy0, wn = x32[0:1].cpu().numpy(), dy32[0:1].cpu().numpy(), w.cpu().numpy()
    errs = {}
    for name in ("fp32", "bf16"):
        x, dy, y, dx, dw = res[name]
        gy = y[0:1].reshape(-1)[idx.to(dev)].double().cpu().numpy()
        gdx = dx[0:1].reshape(-1)[idx.to(dev)].double().cpu().numpy()
        xin, dyin = (x0, dy0) if name == "fp32" else (xb0, dyb0)
        e = {"y": _normwise(gy, oracle.dw_fwd_points(xin, wn, 0, idx.numpy())),
             "dx": _normwise(gdx, oracle.dw_bwd_input_points(dyin, wn, 0, idx.numpy()))}
        if name == "bf16":
            e["y_vs_fp32_inputs"] = _normwise(gy, oracle.dw_fwd_points(x0, wn, 0, idx.numpy()))
            e["dx_vs_fp32_inputs"] = _normwise(gdx, oracle.dw_bwd_input_points(dy0, wn, 0,
                                                                                idx.numpy()))
        errs[name] = e
    out["fp32"]["err_normwise_sampled"] = errs["fp32"]
    out["bf16"]["err_normwise_sampled"] = errs["bf16"]
    out["bf16_over_fp32"] = out["bf16"]["value"] / out["fp32"]["value"]
    out["workload"] = f"{Nb}x3x2048x2048, K=9 normal(0,0.1), zero border, fwd+bwd"
    # K = 9 is past the FP32 ridge (both storage types are ALU-bound); the same
    # images with a 3 x 3 filter are HBM-bound, where halving the bytes pays.
    del res
    k3 = {}
    w3 = (torch.randn((Cb, 3, 3), generator=torch.Generator().manual_seed(2509)) * 0.1).to(dev)
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        x, dy = x32.to(dt), dy32.to(dt)
        y, dx = torch.empty_like(x), torch.empty_like(x)
        dw = torch.empty((Cb, 3, 3), device=dev)
        d = L.desc(Nb, Cb, Cb, Hb, Wb, 3, Cb, 0, L.GIGA_F32 if dt == torch.float32 else L.GIGA_BF16,
                   L.GIGA_LAYOUT_NCHW)
        wsb = L.giga_conv2d_workspace_size(d, 6)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        if tune:
            L.check(L.giga_autotune_conv2d(d, 7, x.data_ptr(), w3.data_ptr(), y.data_ptr(),
                                           dy.data_ptr(), dx.data_ptr(), dw.data_ptr(),
                                           ws.data_ptr(), wsb, sp), "autotune")

        def run3():
            L.check(L.giga_conv2d_fwd(d, x.data_ptr(), w3.data_ptr(), y.data_ptr(), None, 0, sp),
                    "fwd")
            L.check(L.giga_conv2d_bwd(d, x.data_ptr(), dy.data_ptr(), w3.data_ptr(), dx.data_ptr(),
                                      dw.data_ptr(), ws.data_ptr(), wsb, sp), "bwd")
        k3[name + "_ms"] = _events(stream, run3, iters)
        del x, dy, y, dx, ws
    k3["bf16_over_fp32"] = k3["fp32_ms"] / k3["bf16_ms"]
    k3["workload"] = f"{Nb}x3x2048x2048, K=3 normal(0,0.1), zero border, fwd+bwd (HBM-bound)"
    out["k3"] = k3
    return out


def compare_ragged(dev, iters):
    """256 ragged 3-channel images (H, W uniform in [64, 4096], K in {3,5,9,11}),
    zero border, fwd + both gradients: one persistent launch replayed from a CUDA
    graph vs a loop of per-image FP32 calls on the same GPU."""
    import torch
    import workloads
    import paper_2504_01266_gb300 as giga
    from paper_2504_01266_gb300 import _lib as L
    shapes = workloads.ragged_shapes()[:RAGGED_IMAGES]
    imgs, taps = [], 0
    for idx, (h, w_, k) in enumerate(shapes):
        g = workloads.generator("ragged", salt=idx + 1, device=str(dev))
        x = torch.rand((3, h, w_), generator=g, device=dev)
        wt = torch.randn((3, k, k), generator=g, device=dev) * 0.1
        dy = torch.randn((3, h, w_), generator=g, device=dev)
        imgs.append({"x": x, "dy": dy, "w": wt, "y": torch.empty_like(x),
                     "dx": torch.empty_like(x), "dw": torch.empty((3, k, k), device=dev)})
        taps += 3 * 3 * h * w_ * k * k
    stream = torch.cuda.current_stream(dev)
    plan = giga.BatchedPlan(imgs, 7, "zero")
    plan.upload()
    tpc = plan.autotune()   # tiles per chunk of the persistent launch, before capture
    torch.cuda.synchronize(dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
    torch.cuda.synchronize(dev)
    ms_graph = _events(stream, graph.replay, iters)
    sp = stream.cuda_stream
    descs = [L.desc(1, 3, 3, im["x"].shape[1], im["x"].shape[2], im["w"].shape[-1], 3, 0,
                    L.GIGA_F32, L.GIGA_LAYOUT_NCHW) for im in imgs]
    wsb = max(L.giga_conv2d_workspace_size(d, 6) for d in descs)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ref_dy = [im["dx"].clone() for im in imgs[:4]]
    ref_y = [im["y"].clone() for im in imgs[:4]]

    def loop():
        for d, im in zip(descs, imgs):
            L.check(L.giga_conv2d_fwd(d, im["x"].data_ptr(), im["w"].data_ptr(),
                                      im["y"].data_ptr(), None, 0, sp), "fwd")
            L.check(L.giga_conv2d_bwd(d, im["x"].data_ptr(), im["dy"].data_ptr(),
                                      im["w"].data_ptr(), im["dx"].data_ptr(),
                                      im["dw"].data_ptr(), ws.data_ptr(), wsb, sp), "bwd")
    ms_loop = _events(stream, loop, max(2, iters // 2))
    same = all(torch.equal(a, im["y"]) and torch.equal(b, im["dx"])
               for a, b, im in zip(ref_y, ref_dy, imgs[:4]))
    plan.close()
    px = sum(3 * h * w_ for h, w_, _ in shapes)
    return {"workload": f"{len(shapes)} images 3 x U[64,4096]^2, K in {{3,5,9,11}}, zero border, "
                        "fwd+bwd",
            "pixels": px, "graph_persistent": {"ms": ms_graph, "value": taps / (ms_graph * 1e-3) / 1e9,
                                               "tiles_per_chunk_autotuned": tpc},
            "per_image_loop": {"ms": ms_loop, "value": taps / (ms_loop * 1e-3) / 1e9,
                               "launches": 4 * len(imgs)},
            "speedup": ms_loop / ms_graph,
            "y_dx_bitwise_equal_to_per_image_path": bool(same)}


def compare_upsample(dev, iters):
    """The paper's sharpening benchmark (Section 6.6) on a 4K image: nearest
    upsampling by 2, 4 and 8, then its 3 x 3 Laplacian (8 surrounded by -1),
    zero border, FP32.  Fused (one pass, the upsampled image never stored) vs
    the two-call path (upsample, then filter), with the output bandwidth of
    the fused pass against the measured HBM peak and sampled errors against
    the FP64 oracle."""
    import torch
    import oracle
    import workloads
    from paper_2504_01266_gb300 import _lib as L
    pk = peaks()
    C, H, W = 3, 2160, 3840
    g = torch.Generator().manual_seed(2504 + 6)
    xh = torch.rand((1, C, H, W), generator=g)
    lap = torch.tensor([[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]).repeat(C, 1, 1)
    x, w = xh.to(dev), lap.to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    d = L.desc(1, C, C, H, W, 3, C, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)
    out = {"workload": "1x3x2160x3840 FP32 (a 4K RGB image), nearest upsampling by s, then "
                       "the paper's 3x3 Laplacian, zero border",
           "scales": {}}
    for s in (2, 4, 8):
        Ho, Wo = H * s, W * s
        y = torch.empty((1, C, Ho, Wo), device=dev)
        up = torch.empty_like(y)
        dbig = L.desc(1, C, C, Ho, Wo, 3, C, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)

        def fused():
            L.check(L.giga_upsample_conv2d_fwd(d, s, x.data_ptr(), w.data_ptr(), y.data_ptr(),
                                               sp), "upsample_conv2d")

        def two_pass():
            L.check(L.giga_upsample_nearest(d, s, x.data_ptr(), up.data_ptr(), sp), "upsample")
            L.check(L.giga_conv2d_fwd(dbig, up.data_ptr(), w.data_ptr(), y.data_ptr(), None, 0,
                                      sp), "fwd")

        def up_only():
            L.check(L.giga_upsample_nearest(d, s, x.data_ptr(), up.data_ptr(), sp), "upsample")
        t_fused = _events(stream, fused, iters)
        t_two = _events(stream, two_pass, iters)
        t_up = _events(stream, up_only, iters)
        fused()
        px = C * Ho * Wo
        bytes_fused = 4 * px + 4 * C * H * W   # write y, read x once
        gbs = bytes_fused / (t_fused * 1e-3) / 1e9
        idx = torch.unique(torch.cat([workloads.sample_indices(px, 1500, salt=s),
                                      workloads.border_indices(1, C, Ho, Wo, 2, salt=s)]))
        got = y.reshape(-1)[idx.to(dev)].double().cpu().numpy()
        ref = oracle.upsample_dw_fwd_points(xh.numpy(), lap.numpy(), 0, s, idx.numpy())
        out["scales"][str(s)] = {
            "fused_ms": t_fused, "two_pass_ms": t_two, "upsample_only_ms": t_up,
            "speedup": t_two / t_fused, "output_gpixel_s": px / (t_fused * 1e-3) / 1e9,
            "fused_gbs": gbs, "fused_frac_of_hbm": gbs / pk["hbm_gbs"],
            "err_normwise_sampled": _normwise(got, ref)}
        del y, up
        torch.cuda.empty_cache()
    return out


def compare_up_batched(dev, iters):
    """The sharpening benchmark over a database of images (Sections 5 and 6.6):
    128 RGB FP32 images, sides uniform in [64, 1024], each upsampled by its own
    scale (2-8) and filtered with its own K x K filters (K in {3, 5, 9, 11}),
    zero border.  The batched path (one launch per filter size, 4 here) replayed
    from a CUDA graph vs a loop of single-image fused calls (one launch per
    image) on the same GPU, with the batched path's output bandwidth and FP32
    FMA rate against their peaks and sampled errors against the oracle."""
    import torch
    import numpy as np
    import oracle
    import workloads
    import paper_2504_01266_gb300 as giga
    from paper_2504_01266_gb300 import _lib as L
    pk = peaks()
    shapes = workloads.up_ragged_shapes()[:RAGGED_IMAGES]
    host, imgs = [], []
    for i, (h, w_, s, k) in enumerate(shapes):
        x, w = workloads.up_ragged_image(i, h, w_, k)
        host.append((x, w, s))
        imgs.append({"x": x.to(dev), "w": w.to(dev), "scale": s,
                     "y": torch.empty((3, h * s, w_ * s), device=dev)})
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    plan = giga.UpsampleBatchedPlan(imgs, "zero")
    plan.upload()
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.run()
    torch.cuda.synchronize(dev)
    ms_graph = _events(stream, graph.replay, iters)
    graph.replay()
    torch.cuda.synchronize(dev)
    first = [im["y"].reshape(-1)[:4096].clone() for im in imgs[:8]]
    descs = [L.desc(1, 3, 3, h, w_, k, 3, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)
             for h, w_, s, k in shapes]

    def loop():
        for d, im in zip(descs, imgs):
            L.check(L.giga_upsample_conv2d_fwd(d, im["scale"], im["x"].data_ptr(),
                                               im["w"].data_ptr(), im["y"].data_ptr(), sp),
                    "upsample_conv2d")
    ms_loop = _events(stream, loop, max(2, iters // 2))
    same = all(torch.equal(a, im["y"].reshape(-1)[:4096]) for a, im in zip(first, imgs[:8]))
    plan.close()
    # sampled outputs of every 8th image against the oracle
    worst = 0.0
    for i in range(0, len(shapes), 8):
        x, w, s = host[i]
        y = imgs[i]["y"]
        idx = workloads.sample_indices(y.numel(), 300, salt=300 + i)
        got = y.reshape(-1)[idx.to(dev)].double().cpu().numpy()
        ref = oracle.upsample_dw_fwd_points(x.numpy()[None], w.numpy(), 0, s, idx.numpy())
        worst = max(worst, _normwise(got, ref))
    px = sum(3 * h * w_ * s * s for h, w_, s, _ in shapes)
    fma = sum(3 * h * w_ * s * s * k * k for h, w_, s, k in shapes)
    nbytes = sum(4 * 3 * h * w_ * (s * s + 1) for h, w_, s, _ in shapes)   # write y, read x
    gbs = nbytes / (ms_graph * 1e-3) / 1e9
    tflops = 2 * fma / (ms_graph * 1e-3) / 1e12
    del imgs, graph
    torch.cuda.empty_cache()
    return {"workload": f"{len(shapes)} RGB FP32 images, sides U[64,1024], per-image scale "
                        "U{2..8} and KxK filters K in {3,5,9,11} normal(0,0.1), zero border",
            "output_pixels": px, "gpixel_tap_s": fma / (ms_graph * 1e-3) / 1e9,
            "graph_batched": {"ms": ms_graph, "launches": len({k for *_, k in shapes}),
                              "gbs": gbs, "frac_of_hbm": gbs / pk["hbm_gbs"],
                              "tflops": tflops, "frac_of_fp32": tflops / pk["fp32_tflops"]},
            "per_image_loop": {"ms": ms_loop, "launches": len(shapes)},
            "speedup": ms_loop / ms_graph, "equal_to_single_image_path": bool(same),
            "err_normwise_sampled": worst}


def compare_separable(dev, iters):
    """Separable filters (Gaussians, sigma = K / 6) on the benchmark images
    (8 x 3 x 4096 x 4096 FP32, clamp): the row-then-column path vs the general
    K x K forward on the same outer-product filter, with the separable path's
    HBM fraction (8 bytes per pixel) and sampled errors against the oracle."""
    import torch
    import numpy as np
    import oracle
    import workloads
    from paper_2504_01266_gb300 import _lib as L
    pk = peaks()
    x, _ = workloads.plain_scale(3, N=N)
    xd = x.to(dev)
    y = torch.empty_like(xd)
    Nn, Cc, Hh, Ww = x.shape
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    out = {"workload": f"{N}x3x4096x4096 FP32 U[0,1), Gaussian filters sigma = K/6 (row and "
                       "column factors), clamp border", "K": {}}
    for K in (3, 7, 15):
        r = K // 2
        t = np.exp(-np.arange(-r, r + 1) ** 2 / (2.0 * (K / 6.0) ** 2))
        t = (t / t.sum()).astype(np.float32)
        f = torch.from_numpy(np.repeat(t[None], Cc, 0)).to(dev)
        wfull = (f[:, :, None] * f[:, None, :]).contiguous()
        d = L.desc(Nn, Cc, Cc, Hh, Ww, K, Cc, 1, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)

        def sep():
            L.check(L.giga_conv2d_fwd_separable(d, xd.data_ptr(), f.data_ptr(), f.data_ptr(),
                                                y.data_ptr(), sp), "separable")

        def full():
            L.check(L.giga_conv2d_fwd(d, xd.data_ptr(), wfull.data_ptr(), y.data_ptr(), None, 0,
                                      sp), "fwd")
        t_full = _events(stream, full, iters)
        t_sep = _events(stream, sep, iters)
        sep()
        idx = workloads.sample_indices(x.numel(), 1500, salt=70 + K)
        got = y.reshape(-1)[idx.to(dev)].double().cpu().numpy()
        ref = oracle.dw_fwd_points(x.numpy(), (np.outer(t, t)[None].repeat(Cc, 0)).astype(np.float64),
                                   1, idx.numpy())
        gbs = 8 * x.numel() / (t_sep * 1e-3) / 1e9
        out["K"][str(K)] = {"separable_ms": t_sep, "full_ms": t_full, "speedup": t_full / t_sep,
                            "separable_gbs": gbs, "separable_frac_of_hbm": gbs / pk["hbm_gbs"],
                            "gpixel_tap_s": x.numel() * K * K / (t_sep * 1e-3) / 1e9,
                            "err_normwise_sampled": _normwise(got, ref)}
    del xd, y
    torch.cuda.empty_cache()
    return out


def compare_gray(dev, iters):
    """Grayscale then filter (Sections 4.2.5, 4.2.4) on 8 RGB images of
    4096 x 4096 FP32 with the paper's 3 x 3 Laplacian, zero border: the fused
    pass (gray formed in shared memory) vs the two calls (convert, then
    filter), with the fused pass's HBM fraction (12 bytes read + 4 written per
    gray pixel) and sampled errors against the oracle."""
    import torch
    import oracle
    import workloads
    from paper_2504_01266_gb300 import _lib as L
    pk = peaks()
    x, _ = workloads.plain_scale(3, N=N)     # N x 3 x 4096 x 4096, read as R, G, B
    xd = x.to(dev)
    Nn, _, Hh, Ww = x.shape
    lap = torch.tensor([[[-1.0, -1, -1], [-1, 8, -1], [-1, -1, -1]]], device=dev)
    y = torch.empty((Nn, 1, Hh, Ww), device=dev)
    g = torch.empty_like(y)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    d = L.desc(Nn, 3, 1, Hh, Ww, 3, 1, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)
    dg = L.desc(Nn, 1, 1, Hh, Ww, 3, 1, 0, L.GIGA_F32, L.GIGA_LAYOUT_NCHW)

    def fused():
        L.check(L.giga_gray_conv2d_fwd(d, xd.data_ptr(), lap.data_ptr(), y.data_ptr(), sp), "gray")

    def two():
        L.check(L.giga_rgb_to_gray(d, xd.data_ptr(), g.data_ptr(), sp), "rgb_to_gray")
        L.check(L.giga_conv2d_fwd(dg, g.data_ptr(), lap.data_ptr(), y.data_ptr(), None, 0, sp),
                "fwd")
    t_two = _events(stream, two, iters)
    t_fused = _events(stream, fused, iters)
    fused()
    idx = workloads.sample_indices(y.numel(), 1500, salt=81)
    got = y.reshape(-1)[idx.to(dev)].double().cpu().numpy()
    flat = idx.numpy()
    n_img, rest = flat // (Hh * Ww), flat % (Hh * Ww)
    ref = []
    for n in sorted(set(n_img.tolist())):
        sel = n_img == n
        gray = oracle.rgb_to_gray(x[n:n + 1].numpy())
        ref.append((sel, oracle.dw_fwd_points(gray, lap.cpu().numpy(), 0, rest[sel])))
    refv = got.copy()
    for sel, vals in ref:
        refv[sel] = vals
    gbs = 16 * Nn * Hh * Ww / (t_fused * 1e-3) / 1e9
    del xd, y, g
    torch.cuda.empty_cache()
    return {"workload": f"{N} RGB images 3x4096x4096 FP32, paper's 3x3 Laplacian on the gray "
                        "image, zero border",
            "fused_ms": t_fused, "two_pass_ms": t_two, "speedup": t_two / t_fused,
            "fused_gbs": gbs, "fused_frac_of_hbm": gbs / pk["hbm_gbs"],
            "err_normwise_sampled": _normwise(got, refv)}


def compare_dense(dev, iters, bf16_peak):
    """Dense 3 x 3, 64 -> 64 channels, 8 x 1024 x 1024 BF16 NHWC on tcgen05:
    forward, input gradient and filter gradient, TFLOP/s against the measured
    BF16 peak, sampled error against the FP64 oracle."""
    import torch
    import oracle
    import workloads
    import paper_2504_01266_gb300 as giga
    x, w, dy = workloads.dense()
    xc, wc, dyc = x.to(dev), w.to(dev), dy.to(dev)
    stream = torch.cuda.current_stream(dev)
    y = torch.empty_like(xc)
    dx = torch.empty_like(dyc)
    dw = torch.empty((64, 3, 3, 64), device=dev)
    flop = 2 * 8 * 1024 * 1024 * 64 * 64 * 9
    res = {}
    for name, fn in (("fwd", lambda: giga.dense_conv2d_fwd(xc, wc, out=y)),
                     ("bwd_input", lambda: giga.dense_conv2d_bwd_input(dyc, wc, out=dx)),
                     ("bwd_filter", lambda: giga.dense_conv2d_bwd_filter(xc, dyc, out=dw))):
        ms = _events(stream, fn, iters)
        tf = flop / (ms * 1e-3) / 1e12
        res[name] = {"ms": ms, "tflops": tf, "frac_of_bf16_peak": tf / bf16_peak}
    giga.check_device_error(dev)
    idx = workloads.sample_indices(y.numel(), 1500, salt=11)
    got = y.reshape(-1)[idx.to(dev)].double().cpu().numpy()
    ref = oracle.dense_fwd_points(x.double().numpy(), w.double().numpy(), 0, idx.numpy())
    res["fwd"]["err_normwise_sampled"] = _normwise(got, ref)
    res["workload"] = "8x1024x1024x64 BF16 NHWC, 3x3 64->64 normal(0,0.05), zero border"
    res["bytes_per_op"] = 2 * x.numel() * 2
    return res


# ------------------------------------------------------------------- GPU

def check_step(dev, x, dy, filt, run_k, n_points=1500, n_taps=6):
    """Errors of the timed step's own outputs against the FP64 oracle.

    For every K the step's forward and backward calls are repeated once in
    the timed launch configuration (y and dx are shared by the three filter
    sizes, so each K's outputs are checked right after its own calls).
    Sampled y and dx pixels of the first and last image (every kind of border
    pixel included) and `n_taps` filter-gradient taps per K (corners, centre,
    seeded others; each a sum over the whole batch) are compared with the
    oracle; returns {K: {"y", "dx", "dw"}} normwise errors over the samples."""
    import numpy as np
    import torch
    import oracle
    import workloads
    Nn, Cc, Hh, Ww = x.shape
    imgs = sorted({0, Nn - 1})
    x64 = x.cpu().numpy().astype(np.float64)
    dy64 = dy.cpu().numpy().astype(np.float64)
    xs, dys = np.ascontiguousarray(x64[imgs]), np.ascontiguousarray(dy64[imgs])
    plane = Cc * Hh * Ww
    # rows and columns 1..7 from each edge: their reads (forward) or the
    # contributions they receive (input gradient) cross the border
    g = np.random.default_rng(2521)
    near = []
    for p in range(len(imgs) * Cc):
        i, j = int(g.integers(0, Hh)), int(g.integers(0, Ww))
        for d in range(1, 8):
            near += [p * Hh * Ww + d * Ww + j, p * Hh * Ww + (Hh - 1 - d) * Ww + j,
                     p * Hh * Ww + i * Ww + d, p * Hh * Ww + i * Ww + Ww - 1 - d]
    sub = torch.unique(torch.cat([
        workloads.sample_indices(len(imgs) * plane, n_points, salt=21),
        workloads.border_indices(len(imgs), Cc, Hh, Ww, per_plane=2, salt=21),
        torch.tensor(near, dtype=torch.int64)]))
    full = (torch.tensor(imgs)[sub // plane] * plane + sub % plane).to(dev)
    out = {}
    for K in KS:
        y, dx, dw = run_k(K)
        torch.cuda.synchronize(dev)
        w = filt[K].double().cpu().numpy()
        gy = y.reshape(-1)[full].double().cpu().numpy()
        gdx = dx.reshape(-1)[full].double().cpu().numpy()
        ry = oracle.dw_fwd_points(xs, w, oracle.CLAMP, sub.numpy())
        rdx = oracle.dw_bwd_input_points(dys, w, oracle.CLAMP, sub.numpy())
        kk = K * K
        rng = np.random.default_rng(2504 + K)
        taps = sorted({0, kk // 2, kk - 1, *(c * kk + int(t) for c, t in
                                              zip(rng.integers(0, Cc, n_taps - 3),
                                                  rng.integers(0, kk, n_taps - 3)))})
        rdw = oracle.dw_bwd_filter_taps(x64, dy64, K, oracle.CLAMP, np.array(taps))
        gdw = dw.reshape(-1)[torch.tensor(taps, device=dev)].double().cpu().numpy()
        out[K] = {"y": _normwise(gy, ry), "dx": _normwise(gdx, rdx), "dw": _normwise(gdw, rdw),
                  "points": int(sub.numel()), "taps": len(taps)}
    del x64, dy64
    return out


def summarize_checks(checks):
    """Per-K sampled errors of the timed step, compact, with the verdict
    against the FP32 tolerance (1e-5 normwise)."""
    if not checks:
        return None
    worst = max(max(c["y"], c["dx"], c["dw"]) for c in checks.values())
    out = {f"K{K}": _r([c["y"], c["dx"], c["dw"]], 2) for K, c in checks.items()}
    out["order"] = "err_normwise_sampled y, dx, dw vs the FP64 oracle"
    out["ok"] = bool(worst <= 1e-5)
    return out


def summarize(compare):
    """The comparisons of the headline metric in a few hundred characters:
    BF16 vs FP32 storage (speed ratio and errors), the ragged persistent
    launch vs the per-image loop, the dense tensor-core case, and the
    widening rows' speed-ups over their unfused forms."""
    if not compare:
        return None
    out = {}
    b = compare.get("bf16")
    if b:
        e16, e32 = b["bf16"]["err_normwise_sampled"], b["fp32"]["err_normwise_sampled"]
        out["bf16_over_fp32"] = {
            "K9": b["bf16_over_fp32"], "K3": b["k3"]["bf16_over_fp32"],
            "ms_K9": [b["bf16"]["ms"], b["fp32"]["ms"]],
            "err_bf16_kernel": [e16["y"], e16["dx"]],
            "err_bf16_e2e": [e16["y_vs_fp32_inputs"], e16["dx_vs_fp32_inputs"]],
            "err_fp32": [e32["y"], e32["dx"]]}
    r = compare.get("ragged")
    if r:
        out["ragged"] = {"graph_ms": r["graph_persistent"]["ms"],
                         "loop_ms": r["per_image_loop"]["ms"], "speedup": r["speedup"],
                         "tpc": r["graph_persistent"]["tiles_per_chunk_autotuned"],
                         "bitwise": r["y_dx_bitwise_equal_to_per_image_path"]}
    d = compare.get("dense")
    if d:
        out["dense"] = {k: [d[k]["tflops"], d[k]["frac_of_bf16_peak"]]
                        for k in ("fwd", "bwd_input", "bwd_filter")}
        out["dense"]["err"] = d["fwd"]["err_normwise_sampled"]
    u = compare.get("upsample_sharpen")
    if u:
        out["upsample_speedup"] = {s: v["speedup"] for s, v in u["scales"].items()}
    ub = compare.get("upsample_sharpen_batched")
    if ub:
        out["up_batched_speedup"] = ub["speedup"]
    sp = compare.get("separable")
    if sp:
        out["separable_speedup"] = {k: v["speedup"] for k, v in sp["K"].items()}
    gr = compare.get("gray_sharpen")
    if gr:
        out["gray_speedup"] = gr["speedup"]
    return _r(out, 3)


def run_giga(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2504_01266_gb300 import _lib, build
    build.build()
    L = _lib
    L.load()
    # the ALU roofline's denominator: this GPU's measured FP32 FMA rate
    measure_fp32_peak(dev)

    g = torch.Generator(device=dev)
    g.manual_seed(2504 + 1)
    x = torch.rand((N, C, H, W), generator=g, device=dev)
    dy = torch.randn((N, C, H, W), generator=g, device=dev)
    ws_cpu = torch.Generator().manual_seed(2505)
    filt = {K: (torch.randn((C, K, K), generator=ws_cpu) * 0.1).to(dev) for K in KS}
    y = torch.empty_like(x)
    dx = torch.empty_like(x)
    dws = {K: torch.empty((C, K, K), device=dev) for K in KS}
    descs = {K: L.desc(N, C, C, H, W, K, C, L.GIGA_BORDER_CLAMP, L.GIGA_F32,
                       L.GIGA_LAYOUT_NCHW) for K in KS}
    ws_bytes = max(L.giga_conv2d_workspace_size(descs[K], L.GIGA_OP_BWD_INPUT |
                                                L.GIGA_OP_BWD_FILTER) for K in KS)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    # per-op events on the launching stream: (K, op) -> list of ms
    op_ms = {(K, op): [] for K in KS for op in ("fwd", "bwd")}

    def step(record=False):
        for K in KS:
            d = descs[K]
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e2 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            L.check(L.giga_conv2d_fwd(d, x.data_ptr(), filt[K].data_ptr(), y.data_ptr(),
                                      None, 0, sp), "fwd")
            if record:
                e1.record(stream)
            L.check(L.giga_conv2d_bwd(d, x.data_ptr(), dy.data_ptr(), filt[K].data_ptr(),
                                      dx.data_ptr(), dws[K].data_ptr(), ws.data_ptr(),
                                      ws_bytes, sp), "bwd")
            if record:
                e2.record(stream)
                op_ms[(K, "fwd")].append((e0, e1))
                op_ms[(K, "bwd")].append((e1, e2))

    # autotune every (K, op) on the real buffers once, outside the timed region
    tuned = {}
    cached = bool(args.tune_cache) and os.path.exists(args.tune_cache)
    if cached:
        L.giga_autotune_set_mode(1)
        L.check(L.giga_autotune_load(args.tune_cache), "giga_autotune_load")
    pinned = args.pin_bwd is not None or args.pin_fwd is not None
    if pinned:
        L.giga_autotune_set_mode(1)
    if not args.no_tune:
        for K in KS:
            d = descs[K]
            if pinned:  # pinned ops use the given candidate, the others their default
                if args.pin_fwd is not None:
                    L.check(L.giga_autotune_set_choice(d, L.GIGA_OP_FWD, args.pin_fwd),
                            "giga_autotune_set_choice")
                if args.pin_bwd is not None:
                    L.check(L.giga_autotune_set_choice(
                        d, L.GIGA_OP_BWD_INPUT | L.GIGA_OP_BWD_FILTER, args.pin_bwd),
                        "giga_autotune_set_choice")
                tuned[K] = {"fwd": L.giga_autotune_choice(d, L.GIGA_OP_FWD),
                            "bwd": L.giga_autotune_choice(d, L.GIGA_OP_BWD_INPUT |
                                                          L.GIGA_OP_BWD_FILTER)}
                continue
            if cached:
                tuned[K] = {"fwd": L.giga_autotune_choice(d, L.GIGA_OP_FWD),
                            "bwd": L.giga_autotune_choice(d, L.GIGA_OP_BWD_INPUT |
                                                          L.GIGA_OP_BWD_FILTER)}
                continue
            L.check(L.giga_autotune_conv2d(d, L.GIGA_OP_FWD | L.GIGA_OP_BWD_INPUT |
                                           L.GIGA_OP_BWD_FILTER, x.data_ptr(),
                                           filt[K].data_ptr(), y.data_ptr(), dy.data_ptr(),
                                           dx.data_ptr(), dws[K].data_ptr(), ws.data_ptr(),
                                           ws_bytes, sp), "autotune")
            tuned[K] = {"fwd": L.giga_autotune_choice(d, L.GIGA_OP_FWD),
                        "bwd": L.giga_autotune_choice(d, L.GIGA_OP_BWD_INPUT |
                                                      L.GIGA_OP_BWD_FILTER)}
        if args.tune_cache and not cached and rank == 0:
            L.check(L.giga_autotune_save(args.tune_cache), "giga_autotune_save")
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    L.giga_launch_count_reset()
    barrier(world)
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index if dev.index is not None else 0) as clocks:
        time.sleep(0.3)  # let the sampler start before the timed region
        t_host0 = time.time()
        start.record(stream)
        for _ in range(args.steps):
            step(record=True)
        end.record(stream)
        torch.cuda.synchronize(dev)
        clocks.mark(t_host0, time.time())
    launches = L.giga_launch_count()
    barrier(world)
    ms_local = start.elapsed_time(end) / args.steps
    rate, ms = aggregate(taps_per_step(), ms_local, world)
    value = rate / 1e9

    # the step's own outputs against the oracle (after timing, same launches)
    checks = None
    if not args.no_check:
        def run_k(K):
            d = descs[K]
            L.check(L.giga_conv2d_fwd(d, x.data_ptr(), filt[K].data_ptr(), y.data_ptr(),
                                      None, 0, sp), "fwd")
            L.check(L.giga_conv2d_bwd(d, x.data_ptr(), dy.data_ptr(), filt[K].data_ptr(),
                                      dx.data_ptr(), dws[K].data_ptr(), ws.data_ptr(),
                                      ws_bytes, sp), "bwd")
            return y, dx, dws[K]
        checks = check_step(dev, x, dy, filt, run_k)

    # per-op roofline from the events recorded inside the timed region
    pk = peaks()
    px = N * C * H * W
    ops = []
    for (K, op), evs in op_ms.items():
        # median over steps: the first op of the first step can include host
        # launch latency (the stream is idle when the timed region starts)
        t = statistics.median(a.elapsed_time(b) for a, b in evs) * 1e-3
        bytes_ = px * (8 if op == "fwd" else 12)
        fma = px * K * K * (1 if op == "fwd" else 2)
        t_hbm = bytes_ / (pk["hbm_gbs"] * 1e9)
        t_alu = 2 * fma / (pk["fp32_tflops"] * 1e12)
        if t_hbm >= t_alu:
            ach, peak, unit, bound, traffic = bytes_ / t / 1e9, pk["hbm_gbs"], "GB/s", "hbm", bytes_
        else:
            ach, peak, unit, bound, traffic = 2 * fma / t / 1e12, pk["fp32_tflops"], "TFLOP/s", "alu", None
        ops.append({"K": K, "op": op, "ms": t * 1e3, "bound": bound, "achieved": ach,
                    "peak": peak, "unit": unit, "frac": ach / peak,
                    "gbs": bytes_ / t / 1e9, "tflops": 2 * fma / t / 1e12})
    # Dominant kernel = largest device time per step.  The forward op is one
    # launch of dw_fwd_kernel; when the backward runs as two passes (tuned
    # candidate 5) that kernel also computes the input gradient, so it runs
    # twice per step; the fused backward is one dw_bwd_kernel launch plus the
    # small fold / finalize launches.
    by = {(o["K"], o["op"]): o for o in ops}
    kernels = []
    for K in KS:
        split = tuned.get(K, {}).get("bwd") == 5
        f, b = by[(K, "fwd")], by[(K, "bwd")]
        kernels.append((f["ms"] * (2 if split else 1), f"dw_fwd_kernel<float,{K},8>", f))
        if not split:
            ring = tuned.get(K, {}).get("bwd") == 6
            kernels.append((b["ms"], f"dw_bwd{'_ring' if ring else ''}_kernel<float,{K}> (with "
                                     "its fold/finalize launches)", b))
        else:
            kernels.append((b["ms"] - f["ms"], f"dw_filter_kernel<float,{K}>", None))
    _, kname, dom = max((k for k in kernels if k[2] is not None), key=lambda k: k[0])
    traffic = None
    if kname in NCU_DRAM_BYTES_PER_PX and (H, W) == (4096, 4096):
        traffic = NCU_DRAM_BYTES_PER_PX[kname] * px
    roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["frac"], "traffic": traffic,
                "kernel": kname, "op": f"{dom['op']} K={dom['K']}",
                "peak_source": (f"{pk['source']} HBM copy" if dom["bound"] == "hbm" else
                                pk["fp32_source"]),
                "sms": pk["sms"], "fp32_tflops_measured": FP32_MEASURED.get("tflops"),
                "fp32_tflops_plain": FP32_MEASURED.get("plain"),
                "fp32x2_tflops_packed": FP32_MEASURED.get("packed"),
                "fp32_tflops_derived": pk["fp32_tflops_derived"]}

    # End to end through the C ABI with host buffers (pinned), copies timed.
    # Every step copies x and dy host->device and reads y, dx and dw of every K
    # back; copies run on their own streams (H2D and D2H engines) and overlap
    # the filtering through events, with the inputs double-buffered.
    e2e = None
    if not args.no_e2e:
        hx = torch.empty((N, C, H, W), pin_memory=True)
        hdy = torch.empty((N, C, H, W), pin_memory=True)
        hx.copy_(x.cpu())
        hdy.copy_(dy.cpu())
        del y, dx
        torch.cuda.empty_cache()
        dx_in = [(x, dy), (torch.empty_like(x), torch.empty_like(dy))]
        outs = {K: (torch.empty_like(x), torch.empty_like(x)) for K in KS}
        hy = {K: torch.empty((N, C, H, W), pin_memory=True) for K in KS}
        hdx = {K: torch.empty((N, C, H, W), pin_memory=True) for K in KS}
        hdw = {K: torch.empty((C, K, K), pin_memory=True) for K in KS}
        s_h2d = torch.cuda.Stream(dev)
        s_d2h = torch.cuda.Stream(dev)
        torch.cuda.synchronize(dev)
        e_steps = max(1, min(args.steps, 5))

        def e2e_pass(n_steps):
            """n_steps pipelined steps; returns device milliseconds for them."""
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            s_h2d.wait_stream(stream)
            s_d2h.wait_stream(stream)
            inputs_free = [torch.cuda.Event(), torch.cuda.Event()]
            for e in inputs_free:
                e.record(stream)
            outs_free = {K: torch.cuda.Event() for K in KS}
            for K in KS:
                outs_free[K].record(stream)
            for it in range(n_steps):
                bx, bdy = dx_in[it % 2]
                s_h2d.wait_event(inputs_free[it % 2])
                with torch.cuda.stream(s_h2d):
                    bx.copy_(hx, non_blocking=True)
                    bdy.copy_(hdy, non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(s_h2d)
                stream.wait_event(loaded)
                for K in KS:
                    yk, dxk = outs[K]
                    stream.wait_event(outs_free[K])
                    d = descs[K]
                    L.check(L.giga_conv2d_fwd(d, bx.data_ptr(), filt[K].data_ptr(),
                                              yk.data_ptr(), None, 0, sp), "fwd")
                    L.check(L.giga_conv2d_bwd(d, bx.data_ptr(), bdy.data_ptr(),
                                              filt[K].data_ptr(), dxk.data_ptr(),
                                              dws[K].data_ptr(), ws.data_ptr(), ws_bytes, sp),
                            "bwd")
                    done = torch.cuda.Event()
                    done.record(stream)
                    s_d2h.wait_event(done)
                    with torch.cuda.stream(s_d2h):
                        hy[K].copy_(yk, non_blocking=True)
                        hdx[K].copy_(dxk, non_blocking=True)
                        hdw[K].copy_(dws[K], non_blocking=True)
                    outs_free[K].record(s_d2h)
                inputs_free[it % 2].record(stream)
            stream.wait_stream(s_d2h)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            return s0.elapsed_time(s1)

        e2e_pass(1)  # untimed: first use of the freshly pinned host buffers
        barrier(world)
        e_total = e2e_pass(e_steps)
        rate, e_ms = aggregate(taps_per_step(), e_total / e_steps, world)
        elem = 4
        e2e = {"value": rate / 1e9, "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": 2 * px * elem,
               "d2h_bytes_per_step": len(KS) * (2 * px * elem) + sum(C * K * K * 4 for K in KS),
               "overlap": "H2D and D2H on separate streams overlapping the filtering"}
        del dx_in, outs, hy, hdx
        torch.cuda.empty_cache()

    compare = None
    if not args.no_compare:
        torch.cuda.empty_cache()
        bf16_peak = 1894.6
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak = float(json.load(f)["bf16_tflops"])
        except Exception:
            pass
        compare = {}
        for name, fn in (("bf16", lambda: compare_bf16(dev, 5)),
                         ("ragged", lambda: compare_ragged(dev, 5)),
                         ("dense", lambda: compare_dense(dev, 10, bf16_peak)),
                         ("upsample_sharpen", lambda: compare_upsample(dev, 10)),
                         ("upsample_sharpen_batched", lambda: compare_up_batched(dev, 5)),
                         ("separable", lambda: compare_separable(dev, 10)),
                         ("gray_sharpen", lambda: compare_gray(dev, 10))):
            compare[name] = fn()
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, dt, desc = oracle_sample_rate(H, 2)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{desc}; {dt:.1f} s"}

    if rank == 0:
        # full per-op and per-comparison detail: stderr (and --detail FILE)
        detail = {"ops": ops, "compare": compare, "checks": checks, "autotune": tuned,
                  "fp32_peak": FP32_MEASURED}
        print("bench detail: " + json.dumps(detail), file=sys.stderr)
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1)
        # the line: contract keys first, then the compact per-op times, the
        # step's own errors and the comparisons, so a tail of the output
        # holds all of the latter
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "C": C, "H": H, "W": W, "K": list(KS),
                       "border": "clamp", "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (1.6 GB per tensor), no flush"},
            "roofline": _r(roofline),
            "cpu_baseline": _r(cpu),
            "e2e": _r(e2e),
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "ops": {f"{o['op']}{o['K']}": _r([o["ms"], o["frac"]], 3) for o in ops},
            "checks": summarize_checks(checks),
            "summary": summarize(compare),
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_section(args):
    import torch
    from paper_2504_01266_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    measure_fp32_peak(dev)
    peak = 1894.6
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    if args.no_tune:
        from paper_2504_01266_gb300 import _lib as L
        L.giga_autotune_set_mode(0)
    fn = {"bf16": lambda: compare_bf16(dev, args.steps, args.bf16_images, not args.no_tune),
          "ragged": lambda: compare_ragged(dev, args.steps),
          "dense": lambda: compare_dense(dev, args.steps, peak),
          "upsample": lambda: compare_upsample(dev, args.steps),
          "up_batched": lambda: compare_up_batched(dev, args.steps),
          "separable": lambda: compare_separable(dev, args.steps),
          "gray": lambda: compare_gray(dev, args.steps)}[args.section]
    print(json.dumps({"section": args.section, "result": fn()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="giga", choices=["giga", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="built-in default configurations")
    ap.add_argument("--pin-bwd", type=int, default=None,
                    help="backward configuration id for every K instead of tuning it "
                         "(0-4: fused kernel, tiles per CTA auto/2/4/8/16; 5: two passes; "
                         "6: persistent kernel with a ring of two or three tile stages)")
    ap.add_argument("--pin-fwd", type=int, default=None,
                    help="forward configuration id for every K instead of tuning it (bits: "
                         "1 = 32-row tiles, 2 = persistent CTAs with a two-stage tile ring, "
                         "4 = L2 prefetch of a later tile)")
    ap.add_argument("--tune-cache", default="",
                    help="autotune cache file: load it and skip tuning if it exists, "
                         "else tune and save the choices there")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the oracle check of the timed step's outputs")
    ap.add_argument("--detail", default="",
                    help="also write the per-op and per-comparison detail to this JSON file")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the BF16 / ragged / dense comparison measurements")
    ap.add_argument("--section",
                    choices=["bf16", "ragged", "dense", "upsample", "up_batched", "separable",
                             "gray"],
                    help="run only this comparison and print its result (profiling aid)")
    ap.add_argument("--ragged-images", type=int, default=None,
                    help="run the ragged comparisons on the first n of their images "
                         "(profiling runs)")
    ap.add_argument("--bf16-images", type=int, default=32,
                    help="images of the BF16 comparison (profiling runs use fewer)")
    ap.add_argument("--images", type=int, default=N,
                    help="images per GPU (profiling runs use 1: 201 MB per tensor, above L2)")
    args = ap.parse_args()
    if args.images != N:
        set_images(args.images)
    if args.ragged_images is not None:
        set_ragged_images(args.ragged_images)
    if args.impl == "reference":
        return run_reference(args)
    if args.section:
        return run_section(args)
    return run_giga(args)


if __name__ == "__main__":
    sys.exit(main())
