"""ctypes binding of libgiga's C ABI (include/giga.h): the same entry-point
names, argument marshalling only.  Every function here forwards plain
integers and device addresses to the library; no arithmetic of the filtering
path happens in Python.

The library must have been built (``python -m paper_2504_01266_gb300.build``);
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgiga.so")

GIGA_OK = 0
GIGA_ERR_INVALID_ARG = 1
GIGA_ERR_UNSUPPORTED = 2
GIGA_ERR_MISALIGNED = 3
GIGA_ERR_WORKSPACE = 4
GIGA_ERR_CUDA = 5
GIGA_ERR_TIMEOUT = 6

GIGA_BORDER_ZERO = 0
GIGA_BORDER_CLAMP = 1
GIGA_F32 = 0
GIGA_BF16 = 1
GIGA_LAYOUT_NCHW = 0
GIGA_LAYOUT_NHWC = 1
GIGA_OP_FWD = 1
GIGA_OP_BWD_INPUT = 2
GIGA_OP_BWD_FILTER = 4

# Every symbol include/giga.h declares (checked by the CPU tests).
EXPORTS = (
    "giga_conv2d_workspace_size", "giga_conv2d_fwd", "giga_conv2d_bwd_input",
    "giga_conv2d_bwd_filter", "giga_conv2d_bwd", "giga_conv2d_bwd_filter_noalloc",
    "giga_conv2d_fwd_separable", "giga_upsample_nearest", "giga_upsample_conv2d_fwd",
    "giga_rgb_to_gray", "giga_gray_conv2d_fwd",
    "giga_batched_plan_create",
    "giga_batched_plan_workspace_size", "giga_batched_plan_upload", "giga_batched_plan_run",
    "giga_batched_plan_destroy", "giga_conv2d_batched", "giga_conv2d_batched_workspace_size",
    "giga_batched_plan_autotune", "giga_batched_plan_tiles_per_chunk",
    "giga_upsample_batched_plan_create", "giga_upsample_batched_plan_workspace_size",
    "giga_upsample_batched_plan_upload", "giga_upsample_batched_plan_run",
    "giga_upsample_batched_plan_destroy", "giga_upsample_conv2d_batched",
    "giga_upsample_conv2d_batched_workspace_size",
    "giga_autotune_set_mode", "giga_autotune_get_mode", "giga_autotune_conv2d",
    "giga_autotune_choice", "giga_autotune_set_choice", "giga_autotune_save",
    "giga_autotune_load", "giga_autotune_clear",
    "giga_status_string", "giga_check_device_error", "giga_selftest_bounded_wait",
    "giga_last_error_detail",
    "giga_launch_count",
    "giga_launch_count_reset",
    "giga_fp32_fma_peak_sink_bytes", "giga_fp32_fma_peak",
)


class giga_conv2d_desc_t(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("C_in", ctypes.c_int64), ("C_out", ctypes.c_int64),
                ("H", ctypes.c_int64), ("W", ctypes.c_int64), ("K", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("border", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class giga_image_t(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("dy", ctypes.c_void_p),
                ("dx", ctypes.c_void_p), ("w", ctypes.c_void_p), ("dw", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("C", ctypes.c_int32),
                ("K", ctypes.c_int32)]


class giga_up_image_t(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("C", ctypes.c_int32),
                ("K", ctypes.c_int32), ("scale", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GigaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {status_string(status)} ({detail})")
        self.status = status


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_DESC = ctypes.POINTER(giga_conv2d_desc_t)
_IMG = ctypes.POINTER(giga_image_t)
_UPIMG = ctypes.POINTER(giga_up_image_t)
_SZ = ctypes.c_size_t
_I32 = ctypes.c_int32
_ST = ctypes.c_int32

_SIGS = {
    "giga_conv2d_workspace_size": (_ST, [_DESC, _I32, ctypes.POINTER(_SZ)]),
    "giga_conv2d_fwd": (_ST, [_DESC, _P, _P, _P, _P, _SZ, _P]),
    "giga_conv2d_bwd_input": (_ST, [_DESC, _P, _P, _P, _P, _SZ, _P]),
    "giga_conv2d_bwd_filter": (_ST, [_DESC, _P, _P, _P, _P, _SZ, _P]),
    "giga_conv2d_bwd": (_ST, [_DESC, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "giga_conv2d_bwd_filter_noalloc": (_ST, [_DESC, _P, _P, _P, _P]),
    "giga_conv2d_fwd_separable": (_ST, [_DESC, _P, _P, _P, _P, _P]),
    "giga_upsample_nearest": (_ST, [_DESC, _I32, _P, _P, _P]),
    "giga_rgb_to_gray": (_ST, [_DESC, _P, _P, _P]),
    "giga_gray_conv2d_fwd": (_ST, [_DESC, _P, _P, _P, _P]),
    "giga_upsample_conv2d_fwd": (_ST, [_DESC, _I32, _P, _P, _P, _P]),
    "giga_batched_plan_create": (_ST, [_IMG, _I32, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    "giga_batched_plan_workspace_size": (_ST, [_P, ctypes.POINTER(_SZ)]),
    "giga_batched_plan_upload": (_ST, [_P, _P, _SZ, _P]),
    "giga_batched_plan_run": (_ST, [_P, _P, _SZ, _P]),
    "giga_batched_plan_destroy": (None, [_P]),
    "giga_batched_plan_autotune": (_ST, [_P, _P, _SZ, _P, ctypes.POINTER(_I32)]),
    "giga_batched_plan_tiles_per_chunk": (_I32, [_P]),
    "giga_conv2d_batched": (_ST, [_IMG, _I32, _I32, _I32, _I32, _P, _SZ, _P]),
    "giga_conv2d_batched_workspace_size": (_ST, [_IMG, _I32, _I32, ctypes.POINTER(_SZ)]),
    "giga_upsample_batched_plan_create": (_ST, [_UPIMG, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    "giga_upsample_batched_plan_workspace_size": (_ST, [_P, ctypes.POINTER(_SZ)]),
    "giga_upsample_batched_plan_upload": (_ST, [_P, _P, _SZ, _P]),
    "giga_upsample_batched_plan_run": (_ST, [_P, _P, _SZ, _P]),
    "giga_upsample_batched_plan_destroy": (None, [_P]),
    "giga_upsample_conv2d_batched": (_ST, [_UPIMG, _I32, _I32, _I32, _P, _SZ, _P]),
    "giga_upsample_conv2d_batched_workspace_size": (_ST, [_UPIMG, _I32, ctypes.POINTER(_SZ)]),
    "giga_autotune_set_mode": (_ST, [_I32]),
    "giga_autotune_get_mode": (_I32, []),
    "giga_autotune_conv2d": (_ST, [_DESC, _I32, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "giga_autotune_choice": (_I32, [_DESC, _I32]),
    "giga_autotune_set_choice": (_ST, [_DESC, _I32, _I32]),
    "giga_autotune_save": (_ST, [ctypes.c_char_p]),
    "giga_autotune_load": (_ST, [ctypes.c_char_p]),
    "giga_autotune_clear": (None, []),
    "giga_status_string": (ctypes.c_char_p, [_ST]),
    "giga_check_device_error": (_ST, [_P]),
    "giga_selftest_bounded_wait": (_ST, [_P]),
    "giga_last_error_detail": (ctypes.c_char_p, []),
    "giga_launch_count": (ctypes.c_uint64, []),
    "giga_launch_count_reset": (None, []),
    "giga_fp32_fma_peak_sink_bytes": (_SZ, []),
    "giga_fp32_fma_peak": (_ST, [_I32, _P, _SZ, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), _P]),
}


def load(path: str | None = None):
    """Load libgiga.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libgiga.so not found at {p}: build it with "
                "`python -m paper_2504_01266_gb300.build` (there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().giga_status_string(status).decode()


def last_error_detail() -> str:
    return load().giga_last_error_detail().decode()


def check(status: int, where: str) -> None:
    if status != GIGA_OK:
        raise GigaError(status, where, last_error_detail())


def desc(N, C_in, C_out, H, W, K, groups, border, dtype, layout) -> giga_conv2d_desc_t:
    return giga_conv2d_desc_t(int(N), int(C_in), int(C_out), int(H), int(W), int(K),
                              int(groups), int(border), int(dtype), int(layout), 0)


# ---- the C ABI, one wrapper per entry point (same names) -----------------

def giga_conv2d_workspace_size(d: giga_conv2d_desc_t, ops: int) -> int:
    n = _SZ(0)
    check(load().giga_conv2d_workspace_size(ctypes.byref(d), ops, ctypes.byref(n)),
          "giga_conv2d_workspace_size")
    return int(n.value)


def giga_conv2d_fwd(d, x, w, y, ws, ws_bytes, stream) -> int:
    return load().giga_conv2d_fwd(ctypes.byref(d), x, w, y, ws, ws_bytes, stream)


def giga_conv2d_bwd_input(d, dy, w, dx, ws, ws_bytes, stream) -> int:
    return load().giga_conv2d_bwd_input(ctypes.byref(d), dy, w, dx, ws, ws_bytes, stream)


def giga_conv2d_bwd_filter(d, x, dy, dw, ws, ws_bytes, stream) -> int:
    return load().giga_conv2d_bwd_filter(ctypes.byref(d), x, dy, dw, ws, ws_bytes, stream)


def giga_conv2d_bwd_filter_noalloc(d, x, dy, dw, stream) -> int:
    return load().giga_conv2d_bwd_filter_noalloc(ctypes.byref(d), x, dy, dw, stream)


def giga_conv2d_bwd(d, x, dy, w, dx, dw, ws, ws_bytes, stream) -> int:
    return load().giga_conv2d_bwd(ctypes.byref(d), x, dy, w, dx, dw, ws, ws_bytes, stream)


def giga_conv2d_fwd_separable(d, x, wcol, wrow, y, stream) -> int:
    return load().giga_conv2d_fwd_separable(ctypes.byref(d), x, wcol, wrow, y, stream)


def giga_rgb_to_gray(d, x, y, stream) -> int:
    return load().giga_rgb_to_gray(ctypes.byref(d), x, y, stream)


def giga_gray_conv2d_fwd(d, x, w, y, stream) -> int:
    return load().giga_gray_conv2d_fwd(ctypes.byref(d), x, w, y, stream)


def giga_upsample_nearest(d, scale, x, y, stream) -> int:
    return load().giga_upsample_nearest(ctypes.byref(d), scale, x, y, stream)


def giga_upsample_conv2d_fwd(d, scale, x, w, y, stream) -> int:
    return load().giga_upsample_conv2d_fwd(ctypes.byref(d), scale, x, w, y, stream)


def giga_batched_plan_create(images, n, ops, border, dtype):
    plan = _P(None)
    check(load().giga_batched_plan_create(images, n, ops, border, dtype, ctypes.byref(plan)),
          "giga_batched_plan_create")
    return plan


def giga_batched_plan_workspace_size(plan) -> int:
    n = _SZ(0)
    check(load().giga_batched_plan_workspace_size(plan, ctypes.byref(n)),
          "giga_batched_plan_workspace_size")
    return int(n.value)


def giga_batched_plan_upload(plan, ws, ws_bytes, stream) -> int:
    return load().giga_batched_plan_upload(plan, ws, ws_bytes, stream)


def giga_batched_plan_run(plan, ws, ws_bytes, stream) -> int:
    return load().giga_batched_plan_run(plan, ws, ws_bytes, stream)


def giga_batched_plan_destroy(plan) -> None:
    load().giga_batched_plan_destroy(plan)


def giga_batched_plan_autotune(plan, ws, ws_bytes, stream) -> int:
    """Returns the chosen tiles per chunk (raises on error)."""
    tpc = _I32(0)
    check(load().giga_batched_plan_autotune(plan, ws, ws_bytes, stream, ctypes.byref(tpc)),
          "giga_batched_plan_autotune")
    return int(tpc.value)


def giga_batched_plan_tiles_per_chunk(plan) -> int:
    return int(load().giga_batched_plan_tiles_per_chunk(plan))


def giga_conv2d_batched(images, n, ops, border, dtype, ws, ws_bytes, stream) -> int:
    return load().giga_conv2d_batched(images, n, ops, border, dtype, ws, ws_bytes, stream)


def giga_conv2d_batched_workspace_size(images, n, ops) -> int:
    size = _SZ(0)
    check(load().giga_conv2d_batched_workspace_size(images, n, ops, ctypes.byref(size)),
          "giga_conv2d_batched_workspace_size")
    return int(size.value)


def giga_upsample_batched_plan_create(images, n, border, dtype):
    plan = _P(None)
    check(load().giga_upsample_batched_plan_create(images, n, border, dtype, ctypes.byref(plan)),
          "giga_upsample_batched_plan_create")
    return plan


def giga_upsample_batched_plan_workspace_size(plan) -> int:
    n = _SZ(0)
    check(load().giga_upsample_batched_plan_workspace_size(plan, ctypes.byref(n)),
          "giga_upsample_batched_plan_workspace_size")
    return int(n.value)


def giga_upsample_batched_plan_upload(plan, ws, ws_bytes, stream) -> int:
    return load().giga_upsample_batched_plan_upload(plan, ws, ws_bytes, stream)


def giga_upsample_batched_plan_run(plan, ws, ws_bytes, stream) -> int:
    return load().giga_upsample_batched_plan_run(plan, ws, ws_bytes, stream)


def giga_upsample_batched_plan_destroy(plan) -> None:
    load().giga_upsample_batched_plan_destroy(plan)


def giga_upsample_conv2d_batched(images, n, border, dtype, ws, ws_bytes, stream) -> int:
    return load().giga_upsample_conv2d_batched(images, n, border, dtype, ws, ws_bytes, stream)


def giga_upsample_conv2d_batched_workspace_size(images, n) -> int:
    size = _SZ(0)
    check(load().giga_upsample_conv2d_batched_workspace_size(images, n, ctypes.byref(size)),
          "giga_upsample_conv2d_batched_workspace_size")
    return int(size.value)


def giga_autotune_set_mode(mode: int) -> None:
    check(load().giga_autotune_set_mode(mode), "giga_autotune_set_mode")


def giga_autotune_get_mode() -> int:
    return int(load().giga_autotune_get_mode())


def giga_autotune_conv2d(d, ops, x, w, y, dy, dx, dw, ws, ws_bytes, stream) -> int:
    return load().giga_autotune_conv2d(ctypes.byref(d), ops, x, w, y, dy, dx, dw, ws, ws_bytes,
                                       stream)


def giga_autotune_choice(d, op) -> int:
    return int(load().giga_autotune_choice(ctypes.byref(d), op))


def giga_autotune_set_choice(d, op, cand) -> int:
    return load().giga_autotune_set_choice(ctypes.byref(d), op, cand)


def giga_autotune_save(path: str) -> int:
    return load().giga_autotune_save(path.encode())


def giga_autotune_load(path: str) -> int:
    return load().giga_autotune_load(path.encode())


def giga_autotune_clear() -> None:
    load().giga_autotune_clear()


def giga_check_device_error(stream) -> int:
    return load().giga_check_device_error(stream)


def giga_selftest_bounded_wait(stream) -> int:
    return load().giga_selftest_bounded_wait(stream)


def giga_launch_count() -> int:
    return int(load().giga_launch_count())


def giga_launch_count_reset() -> None:
    load().giga_launch_count_reset()


def giga_fp32_fma_peak_sink_bytes() -> int:
    return int(load().giga_fp32_fma_peak_sink_bytes())


def giga_fp32_fma_peak(packed, sink, sink_bytes, stream):
    """Measured FP32 FMA throughput: returns (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(load().giga_fp32_fma_peak(packed, sink, sink_bytes, ctypes.byref(tf), ctypes.byref(ms),
                                    stream), "giga_fp32_fma_peak")
    return float(tf.value), float(ms.value)
