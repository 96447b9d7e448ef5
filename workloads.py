"""Seeded synthetic inputs for the filtering workloads.

This module only draws numbers: it holds none of the filtering arithmetic, and
it is the one piece that the oracle tests, the CUDA parity tests and the
benchmark share.  Every tensor comes from a ``torch.Generator`` seeded with
``2504 + workload id`` so that two calls with the same arguments return the
same values on every host.

The six workloads follow the image-filtering workload of the GigaAPI paper
(Section 4.2.4 "Sharpening" and Section 6.6 "API Benchmark #5"): the paper's
photographs are not available, so uniform [0, 1) pixels stand in for them.

  plain_small   1 x 1 x 512 x 512 FP32, one 5 x 5 normalised Gaussian (sigma 1),
                zero border.
  plain_scale   8 x 3 x 4096 x 4096 FP32, depthwise K x K filters normal(0, 0.1)
                for K in {3, 7, 15}, clamp border.
  train         16 x 3 x 2048 x 2048 FP32, 7 x 7 filters normal(0, 0.1),
                upstream gradient normal(0, 1), zero border.
  ragged        256 three-channel images, H and W uniform integers in
                [64, 4096], each with its own filters of size drawn from
                {3, 5, 9, 11}, normal(0, 0.1), zero border.
  bf16          32 x 3 x 2048 x 2048 BF16 images, 9 x 9 filters normal(0, 0.1),
                BF16 upstream gradient normal(0, 1).
  dense         8 x 1024 x 1024 x 64 BF16 NHWC images, 64 x 3 x 3 x 64 BF16
                filters normal(0, 0.05), BF16 upstream gradient normal(0, 1).
  up_ragged     a "photo database" for the sharpening benchmark (Section 6.6
                run over a batch, the goal of Section 5): 128 three-channel
                FP32 images, H and W uniform integers in [64, 1024], each
                upsampled by its own integer scale uniform in [2, 8] and
                filtered with its own filters of size drawn from {3, 5, 9, 11},
                normal(0, 0.1), zero border.

Every generator takes size overrides so that tests can draw the same
distributions at sizes the oracle finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

BASE_SEED = 2504
SEEDS = {"plain_small": 0, "plain_scale": 1, "train": 2, "ragged": 3, "bf16": 4, "dense": 5,
         "up_ragged": 7}


def generator(name: str, salt: int = 0, device: str = "cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(BASE_SEED + SEEDS[name] + 1000 * salt)
    return g


def gaussian_filter(K: int = 5, sigma: float = 1.0) -> torch.Tensor:
    """Normalised K x K Gaussian, built in FP64 and rounded once to FP32."""
    r = (K - 1) // 2
    ax = torch.arange(-r, r + 1, dtype=torch.float64)
    g = torch.exp(-(ax[:, None] ** 2 + ax[None, :] ** 2) / (2.0 * sigma * sigma))
    return (g / g.sum()).to(torch.float32)


def uniform(shape, g: torch.Generator, device="cpu", dtype=torch.float32) -> torch.Tensor:
    return torch.rand(shape, generator=g, device=device, dtype=torch.float32).to(dtype)


def normal(shape, std: float, g: torch.Generator, device="cpu", dtype=torch.float32):
    return (torch.randn(shape, generator=g, device=device, dtype=torch.float32) * std).to(dtype)


def plain_small(H: int = 512, W: int = 512):
    g = generator("plain_small")
    x = uniform((1, 1, H, W), g)
    w = gaussian_filter(5, 1.0).reshape(1, 5, 5)
    return x, w


def plain_scale(K: int, N: int = 8, C: int = 3, H: int = 4096, W: int = 4096,
                device: str = "cpu"):
    """x uniform [0, 1), w normal(0, 0.1) of shape (C, K, K)."""
    g = generator("plain_scale", salt=K, device=device)
    x = uniform((N, C, H, W), g, device)
    w = normal((C, K, K), 0.1, g, device)
    return x, w


def plain_scale_dy(N: int = 8, C: int = 3, H: int = 4096, W: int = 4096, device: str = "cpu"):
    """Upstream gradient of the plain_scale images: normal(0, 1), (N, C, H, W)."""
    g = generator("plain_scale", salt=100, device=device)
    return normal((N, C, H, W), 1.0, g, device)


def train(N: int = 16, C: int = 3, H: int = 2048, W: int = 2048, K: int = 7,
          device: str = "cpu"):
    """x uniform [0, 1), w normal(0, 0.1), dy normal(0, 1)."""
    g = generator("train", device=device)
    x = uniform((N, C, H, W), g, device)
    w = normal((C, K, K), 0.1, g, device)
    dy = normal((N, C, H, W), 1.0, g, device)
    return x, w, dy


@dataclass
class RaggedImage:
    H: int
    W: int
    K: int
    x: torch.Tensor = field(repr=False)
    w: torch.Tensor = field(repr=False)
    dy: torch.Tensor = field(repr=False)


def ragged_shapes(n: int = 256, lo: int = 64, hi: int = 4096, ks=(3, 5, 9, 11)):
    """The (H, W, K) list of the ragged batch, drawn from the workload seed."""
    g = generator("ragged")
    H = torch.randint(lo, hi + 1, (n,), generator=g)
    W = torch.randint(lo, hi + 1, (n,), generator=g)
    Ki = torch.randint(0, len(ks), (n,), generator=g)
    return [(int(h), int(w), int(ks[int(k)])) for h, w, k in zip(H, W, Ki)]


def ragged(n: int = 256, C: int = 3, lo: int = 64, hi: int = 4096, ks=(3, 5, 9, 11),
           device: str = "cpu", dtype=torch.float32):
    """A list of ``RaggedImage``: x (1, C, H, W) uniform, w (C, K, K) normal(0, 0.1),
    dy (1, C, H, W) normal(0, 1); each image draws from its own sub-seed."""
    out = []
    for idx, (h, w_, k) in enumerate(ragged_shapes(n, lo, hi, ks)):
        g = generator("ragged", salt=idx + 1, device=device)
        x = uniform((1, C, h, w_), g, device, dtype)
        w = normal((C, k, k), 0.1, g, device)
        dy = normal((1, C, h, w_), 1.0, g, device, dtype)
        out.append(RaggedImage(h, w_, k, x, w, dy))
    return out


def up_ragged_shapes(n: int = 128, lo: int = 64, hi: int = 1024, scales=(2, 8),
                     ks=(3, 5, 9, 11)):
    """The (H, W, scale, K) list of the upsampling database, drawn from its seed."""
    g = generator("up_ragged")
    H = torch.randint(lo, hi + 1, (n,), generator=g)
    W = torch.randint(lo, hi + 1, (n,), generator=g)
    S = torch.randint(scales[0], scales[1] + 1, (n,), generator=g)
    Ki = torch.randint(0, len(ks), (n,), generator=g)
    return [(int(h), int(w), int(s), int(ks[int(k)])) for h, w, s, k in zip(H, W, S, Ki)]


def up_ragged_image(idx: int, H: int, W: int, K: int, C: int = 3, device: str = "cpu",
                    dtype=torch.float32):
    """Image idx of the upsampling database: x (C, H, W) uniform [0, 1) and
    w (C, K, K) normal(0, 0.1), from the image's own sub-seed."""
    g = generator("up_ragged", salt=idx + 1, device=device)
    x = uniform((C, H, W), g, device, dtype)
    w = normal((C, K, K), 0.1, g, device)
    return x, w


def bf16(N: int = 32, C: int = 3, H: int = 2048, W: int = 2048, K: int = 9,
         device: str = "cpu"):
    """BF16 x uniform [0, 1) and dy normal(0, 1) (drawn in FP32, rounded once),
    FP32 w normal(0, 0.1).  Also returns the FP32 originals of x and dy."""
    g = generator("bf16", device=device)
    x32 = uniform((N, C, H, W), g, device)
    w = normal((C, K, K), 0.1, g, device)
    dy32 = normal((N, C, H, W), 1.0, g, device)
    return x32.to(torch.bfloat16), w, dy32.to(torch.bfloat16), x32, dy32


def dense(N: int = 8, H: int = 1024, W: int = 1024, Ci: int = 64, Co: int = 64, K: int = 3,
          device: str = "cpu"):
    """NHWC BF16 x uniform [0, 1), BF16 w (Co, K, K, Ci) normal(0, 0.05),
    NHWC BF16 dy normal(0, 1)."""
    g = generator("dense", device=device)
    x = uniform((N, H, W, Ci), g, device, torch.bfloat16)
    w = normal((Co, K, K, Ci), 0.05, g, device, torch.bfloat16)
    dy = normal((N, H, W, Co), 1.0, g, device, torch.bfloat16)
    return x, w, dy


def sample_indices(numel: int, count: int, salt: int = 0) -> torch.Tensor:
    """Distinct flat indices in [0, numel), sorted (seeded)."""
    g = torch.Generator()
    g.manual_seed(BASE_SEED + 7919 * (salt + 1))
    count = min(count, numel)
    if numel <= 4 * count:
        return torch.randperm(numel, generator=g)[:count].sort().values
    idx = torch.unique(torch.randint(0, numel, (count + count // 8 + 8,), generator=g))
    return idx[:count]


def border_indices(N: int, C: int, H: int, W: int, per_plane: int = 8, salt: int = 0):
    """Flat NCHW indices that sit on the image edges and corners (where the
    border rule matters), a few per plane."""
    g = torch.Generator()
    g.manual_seed(BASE_SEED + 104729 * (salt + 1))
    out = []
    for n in range(N):
        for c in range(C):
            base = (n * C + c) * H * W
            pts = {(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1)}
            for _ in range(per_plane):
                i = int(torch.randint(0, H, (1,), generator=g))
                j = int(torch.randint(0, W, (1,), generator=g))
                pts.add((0, j)); pts.add((H - 1, j)); pts.add((i, 0)); pts.add((i, W - 1))
            out.extend(base + i * W + j for i, j in sorted(pts))
    return torch.tensor(sorted(set(out)), dtype=torch.int64)
