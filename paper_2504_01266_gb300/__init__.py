"""GB300-native dense 2D image filtering (the sharpening filter of the GigaAPI
paper, Section 4.2.4, widened to K x K depthwise/dense filters, zero/clamp
borders, both gradients, ragged batches and BF16 storage).

PyTorch supplies device memory and streams; every step of the filtering path
runs in libgiga's CUDA kernels behind the C ABI of include/giga.h.  The
helpers below allocate outputs and workspaces with torch and marshal pointers
through ``_lib``.  There is no CPU fallback: calling them without the built
library or without a CUDA tensor raises.

Conventions: depthwise tensors NCHW (FP32 or BF16) with FP32 filters
``w[C][K][K]`` (cross-correlation, tap (a, b) reads pixel (i + a - r, j + b - r));
border "zero" or "clamp".
"""
from __future__ import annotations

import torch

from . import _lib

BORDERS = {"zero": _lib.GIGA_BORDER_ZERO, "clamp": _lib.GIGA_BORDER_CLAMP}
DTYPES = {torch.float32: _lib.GIGA_F32, torch.bfloat16: _lib.GIGA_BF16}

__all__ = ["conv2d", "conv2d_fwd", "conv2d_bwd", "conv2d_bwd_input", "conv2d_bwd_filter",
           "DepthwiseConv2d", "workspace", "BORDERS", "upsample_nearest", "upsample_conv2d",
           "conv2d_separable", "rgb_to_gray", "gray_conv2d", "BatchedPlan",
           "UpsampleBatchedPlan"]


def _border(border) -> int:
    if isinstance(border, str):
        if border not in BORDERS:
            raise ValueError(f"border must be one of {list(BORDERS)}")
        return BORDERS[border]
    return int(border)


def _dtype(t: torch.Tensor) -> int:
    if t.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {t.dtype}: use float32 or bfloat16")
    return DTYPES[t.dtype]


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise RuntimeError("libgiga runs on CUDA tensors only (no CPU fallback)")
        if t is not None and not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def dw_desc(x: torch.Tensor, K: int, border) -> _lib.giga_conv2d_desc_t:
    N, C, H, W = x.shape
    return _lib.desc(N, C, C, H, W, K, C, _border(border), _dtype(x), _lib.GIGA_LAYOUT_NCHW)


def workspace(d: _lib.giga_conv2d_desc_t, ops: int, device) -> torch.Tensor | None:
    n = _lib.giga_conv2d_workspace_size(d, ops)
    if n == 0:
        return None
    return torch.empty(n, dtype=torch.uint8, device=device)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _nbytes(t):
    return 0 if t is None else t.numel()


def conv2d_fwd(x: torch.Tensor, w: torch.Tensor, border="zero", out=None) -> torch.Tensor:
    """y = K_w x (depthwise, NCHW)."""
    _require_cuda(x, w)
    d = dw_desc(x, w.shape[-1], border)
    y = torch.empty_like(x) if out is None else out
    ws = workspace(d, _lib.GIGA_OP_FWD, x.device)
    _lib.check(_lib.giga_conv2d_fwd(d, _ptr(x), _ptr(w), _ptr(y), _ptr(ws), _nbytes(ws),
                                    _stream(x.device)), "giga_conv2d_fwd")
    return y


def conv2d_separable(x: torch.Tensor, wcol: torch.Tensor, wrow: torch.Tensor, border="zero",
                     out=None) -> torch.Tensor:
    """y = K_w x for the separable filter w[c] = outer(wcol[c], wrow[c]) (both
    (C, K) FP32): a row pass then a column pass, 2K multiply-adds per pixel."""
    _require_cuda(x, wcol, wrow)
    d = dw_desc(x, wcol.shape[-1], border)
    y = torch.empty_like(x) if out is None else out
    _lib.check(_lib.giga_conv2d_fwd_separable(d, _ptr(x), _ptr(wcol), _ptr(wrow), _ptr(y),
                                              _stream(x.device)), "giga_conv2d_fwd_separable")
    return y


def _gray_desc(x: torch.Tensor, K: int, border):
    if x.dim() != 4 or x.shape[1] != 3:
        raise ValueError("x must be (N, 3, H, W) with channels R, G, B")
    N, _, H, W = x.shape
    return _lib.desc(N, 3, 1, H, W, K, 1, _border(border), _dtype(x), _lib.GIGA_LAYOUT_NCHW)


def rgb_to_gray(x: torch.Tensor, out=None) -> torch.Tensor:
    """gray = 0.299 R + 0.587 G + 0.114 B: (N, 3, H, W) -> (N, 1, H, W)."""
    _require_cuda(x)
    d = _gray_desc(x, 1, "zero")
    y = torch.empty((x.shape[0], 1) + tuple(x.shape[2:]), dtype=x.dtype, device=x.device) \
        if out is None else out
    _lib.check(_lib.giga_rgb_to_gray(d, _ptr(x), _ptr(y), _stream(x.device)), "giga_rgb_to_gray")
    return y


def gray_conv2d(x: torch.Tensor, w: torch.Tensor, border="zero", out=None) -> torch.Tensor:
    """The filter w (1, K, K) applied to the grayscale image of x, in one pass."""
    _require_cuda(x, w)
    d = _gray_desc(x, w.shape[-1], border)
    y = torch.empty((x.shape[0], 1) + tuple(x.shape[2:]), dtype=x.dtype, device=x.device) \
        if out is None else out
    _lib.check(_lib.giga_gray_conv2d_fwd(d, _ptr(x), _ptr(w), _ptr(y), _stream(x.device)),
               "giga_gray_conv2d_fwd")
    return y


def _up_out(x: torch.Tensor, scale: int, out):
    N, C, H, W = x.shape
    shape = (N, C, H * scale, W * scale)
    if out is None:
        return torch.empty(shape, dtype=x.dtype, device=x.device)
    if tuple(out.shape) != shape:
        raise ValueError(f"out must have shape {shape}")
    return out


def upsample_nearest(x: torch.Tensor, scale: int, out=None) -> torch.Tensor:
    """Nearest-neighbour upsampling by an integer factor (NCHW)."""
    _require_cuda(x)
    d = dw_desc(x, 1, "zero")
    y = _up_out(x, scale, out)
    _lib.check(_lib.giga_upsample_nearest(d, int(scale), _ptr(x), _ptr(y), _stream(x.device)),
               "giga_upsample_nearest")
    return y


def upsample_conv2d(x: torch.Tensor, w: torch.Tensor, scale: int, border="zero",
                    out=None) -> torch.Tensor:
    """The depthwise filter applied to the upsampled image, in one pass."""
    _require_cuda(x, w)
    d = dw_desc(x, w.shape[-1], border)
    y = _up_out(x, scale, out)
    _lib.check(_lib.giga_upsample_conv2d_fwd(d, int(scale), _ptr(x), _ptr(w), _ptr(y),
                                             _stream(x.device)), "giga_upsample_conv2d_fwd")
    return y


def conv2d_bwd_input(dy: torch.Tensor, w: torch.Tensor, border="zero", out=None):
    """dx = K_w^T dy."""
    _require_cuda(dy, w)
    d = dw_desc(dy, w.shape[-1], border)
    dx = torch.empty_like(dy) if out is None else out
    ws = workspace(d, _lib.GIGA_OP_BWD_INPUT, dy.device)
    _lib.check(_lib.giga_conv2d_bwd_input(d, _ptr(dy), _ptr(w), _ptr(dx), _ptr(ws),
                                          _nbytes(ws), _stream(dy.device)),
               "giga_conv2d_bwd_input")
    return dx


def conv2d_bwd_filter(x: torch.Tensor, dy: torch.Tensor, K: int, border="zero", out=None):
    """dw[c][a][b] = sum_{n,i,j} dy * x~ (FP32, shape (C, K, K))."""
    _require_cuda(x, dy)
    d = dw_desc(x, K, border)
    dw = torch.empty((x.shape[1], K, K), dtype=torch.float32, device=x.device) \
        if out is None else out
    ws = workspace(d, _lib.GIGA_OP_BWD_FILTER, x.device)
    _lib.check(_lib.giga_conv2d_bwd_filter(d, _ptr(x), _ptr(dy), _ptr(dw), _ptr(ws),
                                           _nbytes(ws), _stream(x.device)),
               "giga_conv2d_bwd_filter")
    return dw


def conv2d_bwd(x: torch.Tensor, dy: torch.Tensor, w: torch.Tensor, border="zero",
               dx=None, dw=None, ws=None):
    """Both gradients (dx, dw): one fused pass over x and dy, or -- when the
    autotuner chose it for this problem class -- an input-gradient pass and a
    filter-gradient pass."""
    _require_cuda(x, dy, w)
    K = w.shape[-1]
    d = dw_desc(x, K, border)
    dx = torch.empty_like(dy) if dx is None else dx
    dw = torch.empty((x.shape[1], K, K), dtype=torch.float32, device=x.device) \
        if dw is None else dw
    if ws is None:
        ws = workspace(d, _lib.GIGA_OP_BWD_INPUT | _lib.GIGA_OP_BWD_FILTER, x.device)
    _lib.check(_lib.giga_conv2d_bwd(d, _ptr(x), _ptr(dy), _ptr(w), _ptr(dx), _ptr(dw),
                                    _ptr(ws), _nbytes(ws), _stream(x.device)),
               "giga_conv2d_bwd")
    return dx, dw


class DepthwiseConv2d(torch.autograd.Function):
    """Autograd wrapper: forward = giga_conv2d_fwd, backward = the fused
    giga_conv2d_bwd (or one of the two gradients when only one is needed)."""

    @staticmethod
    def forward(ctx, x, w, border="zero"):
        ctx.border = border
        ctx.save_for_backward(x, w)
        return conv2d_fwd(x.contiguous(), w.contiguous(), border)

    @staticmethod
    def backward(ctx, dy):
        x, w = ctx.saved_tensors
        dy = dy.contiguous().to(x.dtype)
        need_x, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dx = dw = None
        if need_x and need_w:
            dx, dw = conv2d_bwd(x, dy, w, ctx.border)
        elif need_x:
            dx = conv2d_bwd_input(dy, w, ctx.border)
        elif need_w:
            dw = conv2d_bwd_filter(x, dy, w.shape[-1], ctx.border)
        return dx, dw, None


def conv2d(x: torch.Tensor, w: torch.Tensor, border="zero") -> torch.Tensor:
    """Depthwise K x K filtering with autograd support."""
    return DepthwiseConv2d.apply(x, w, border)


# ------------------------------------------------------------ ragged batches

class BatchedPlan:
    """One persistent launch over a ragged list of images (giga_batched_plan_*).

    ``images``: list of dicts with device tensors ``x`` / ``y`` / ``dy`` / ``dx``
    of shape (C, H, W) (any subset the ops need) and ``w`` / ``dw`` of shape
    (C, K, K) FP32.  ``ops`` is a GIGA_OP_* bitmask.  ``run()`` is capturable
    into a CUDA graph once ``upload()`` has been issued.
    """

    def __init__(self, images, ops, border="zero", dtype=torch.float32):
        self.n = len(images)
        arr = (_lib.giga_image_t * max(1, self.n))()
        self.keep = []
        for i, im in enumerate(images):
            ref = im.get("x") if im.get("x") is not None else im.get("dy")
            C, H, W = ref.shape[-3:]
            K = im["w"].shape[-1] if im.get("w") is not None else im["dw"].shape[-1]
            _require_cuda(*[im.get(k) for k in ("x", "y", "dy", "dx", "w", "dw")])
            arr[i] = _lib.giga_image_t(
                _ptr(im.get("x")), _ptr(im.get("y")), _ptr(im.get("dy")), _ptr(im.get("dx")),
                _ptr(im.get("w")), _ptr(im.get("dw")), H, W, C, K)
            self.keep.append(im)
        self.arr = arr
        self.ops = ops
        self.plan = _lib.giga_batched_plan_create(arr, self.n, ops, _border(border),
                                                  DTYPES[dtype])
        self.ws_bytes = _lib.giga_batched_plan_workspace_size(self.plan)
        dev = ref.device if self.n else torch.device("cuda")
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.device = dev

    def upload(self):
        _lib.check(_lib.giga_batched_plan_upload(self.plan, self.ws.data_ptr(), self.ws.numel(),
                                                 _stream(self.device)),
                   "giga_batched_plan_upload")

    def run(self):
        _lib.check(_lib.giga_batched_plan_run(self.plan, self.ws.data_ptr(), self.ws.numel(),
                                              _stream(self.device)),
                   "giga_batched_plan_run")

    def autotune(self) -> int:
        """Time the launch at 1 to 32 tiles per chunk (powers of 2) on these buffers
        (outputs overwritten), keep the fastest; returns it.  Not capturable."""
        return _lib.giga_batched_plan_autotune(self.plan, self.ws.data_ptr(), self.ws.numel(),
                                               _stream(self.device))

    @property
    def tiles_per_chunk(self) -> int:
        return _lib.giga_batched_plan_tiles_per_chunk(self.plan)

    def close(self):
        if self.plan:
            _lib.giga_batched_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UpsampleBatchedPlan:
    """Upsample-then-filter over a ragged list of images in one persistent launch
    (giga_upsample_batched_plan_*).

    ``images``: list of dicts with device tensors ``x`` (C, H, W), ``y``
    (C, H * scale, W * scale) in the same dtype, ``w`` (C, K, K) FP32 and an
    integer ``scale`` >= 2.  ``run()`` is capturable into a CUDA graph once
    ``upload()`` has been issued.
    """

    def __init__(self, images, border="zero", dtype=torch.float32):
        self.n = len(images)
        arr = (_lib.giga_up_image_t * max(1, self.n))()
        self.keep = []
        dev = torch.device("cuda")
        for i, im in enumerate(images):
            C, H, W = im["x"].shape[-3:]
            _require_cuda(im["x"], im["y"], im["w"])
            arr[i] = _lib.giga_up_image_t(_ptr(im["x"]), _ptr(im["y"]), _ptr(im["w"]), H, W, C,
                                          im["w"].shape[-1], int(im["scale"]), 0)
            self.keep.append(im)
            dev = im["x"].device
        self.arr = arr
        self.plan = _lib.giga_upsample_batched_plan_create(arr, self.n, _border(border),
                                                           DTYPES[dtype])
        self.ws_bytes = _lib.giga_upsample_batched_plan_workspace_size(self.plan)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.device = dev

    def upload(self):
        _lib.check(_lib.giga_upsample_batched_plan_upload(self.plan, self.ws.data_ptr(),
                                                          self.ws.numel(), _stream(self.device)),
                   "giga_upsample_batched_plan_upload")

    def run(self):
        _lib.check(_lib.giga_upsample_batched_plan_run(self.plan, self.ws.data_ptr(),
                                                       self.ws.numel(), _stream(self.device)),
                   "giga_upsample_batched_plan_run")

    def close(self):
        if self.plan:
            _lib.giga_upsample_batched_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ dense 3 x 3

def dense_desc(x: torch.Tensor, K: int = 3, border="zero") -> _lib.giga_conv2d_desc_t:
    N, H, W, C = x.shape
    return _lib.desc(N, C, C, H, W, K, 1, _border(border), _dtype(x), _lib.GIGA_LAYOUT_NHWC)


def dense_conv2d_fwd(x: torch.Tensor, w: torch.Tensor, out=None) -> torch.Tensor:
    """Dense 3 x 3 filter, 64 -> 64 channels, BF16 NHWC, zero border (tcgen05).
    x (N, H, W, 64), w (64, 3, 3, 64) = [C_out][K][K][C_in]."""
    _require_cuda(x, w)
    d = dense_desc(x, w.shape[1])
    y = torch.empty_like(x) if out is None else out
    _lib.check(_lib.giga_conv2d_fwd(d, _ptr(x), _ptr(w), _ptr(y), None, 0, _stream(x.device)),
               "giga_conv2d_fwd (dense)")
    return y


def dense_conv2d_bwd_input(dy: torch.Tensor, w: torch.Tensor, out=None) -> torch.Tensor:
    _require_cuda(dy, w)
    d = dense_desc(dy, w.shape[1])
    dx = torch.empty_like(dy) if out is None else out
    ws = workspace(d, _lib.GIGA_OP_BWD_INPUT, dy.device)
    _lib.check(_lib.giga_conv2d_bwd_input(d, _ptr(dy), _ptr(w), _ptr(dx), _ptr(ws), _nbytes(ws),
                                          _stream(dy.device)), "giga_conv2d_bwd_input (dense)")
    return dx


def check_device_error(device=None) -> None:
    """Raise if a pipelined tensor-core kernel reported an expired wait."""
    dev = torch.device("cuda") if device is None else device
    _lib.check(_lib.giga_check_device_error(_stream(dev)), "giga_check_device_error")


def dense_conv2d_bwd_filter(x: torch.Tensor, dy: torch.Tensor, out=None) -> torch.Tensor:
    """Filter gradient of the dense 3 x 3 filter: FP32 (64, 3, 3, 64)."""
    _require_cuda(x, dy)
    d = dense_desc(x, 3)
    dw = torch.empty((64, 3, 3, 64), dtype=torch.float32, device=x.device) if out is None else out
    ws = workspace(d, _lib.GIGA_OP_BWD_FILTER, x.device)
    _lib.check(_lib.giga_conv2d_bwd_filter(d, _ptr(x), _ptr(dy), _ptr(dw), _ptr(ws), _nbytes(ws),
                                           _stream(x.device)), "giga_conv2d_bwd_filter (dense)")
    return dw
