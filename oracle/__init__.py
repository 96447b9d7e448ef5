"""FP64 CPU oracle for dense 2D image filtering -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never touches the CUDA library: the two share no code.

The arithmetic lives in ``giga_oracle.c`` (plain C, double precision): the
neighbourhood sum of the GigaAPI paper, Section 4.2.4 ("Sharpening"), widened
to odd K x K depthwise filters, zero or clamp borders, the two gradients and
the dense multi-channel case.  This module compiles it with gcc and wraps it
with ctypes; every wrapper takes numpy arrays (any float dtype, converted to
float64) and returns float64 arrays.

Conventions: depthwise tensors are NCHW with filters ``w[C][K][K]``; dense
tensors are NHWC with filters ``w[Co][K][K][Ci]``; tap ``(a, b)`` reads the
neighbour at ``(i + a - r, j + b - r)`` with ``r = (K - 1) // 2``
(cross-correlation).  ``border`` is 0 (zero) or 1 (clamp).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

ZERO = 0
CLAMP = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "giga_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I64 = ctypes.c_int64
_INT = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile ``giga_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, OpenMP).

    ``-ffp-contract=off`` keeps every multiply and add a separate IEEE double
    operation on every host architecture.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        six = [_I64, _I64, _I64, _I64, _INT, _INT]          # N, C, H, W, K, border
        dense = [_I64, _I64, _I64, _I64, _I64, _INT, _INT]  # N, H, W, Ci, Co, K, border
        sigs = {
            "oracle_dw_fwd": [_D, _D, _D] + six,
            "oracle_dw_fwd_points": [_D, _D] + six + [_I64P, _I64, _D],
            "oracle_dw_bwd_input": [_D, _D, _D] + six,
            "oracle_dw_bwd_input_points": [_D, _D] + six + [_I64P, _I64, _D],
            "oracle_dw_bwd_filter": [_D, _D, _D] + six,
            "oracle_dw_bwd_filter_taps": [_D, _D] + six + [_I64P, _I64, _D],
            "oracle_dense_fwd": [_D, _D, _D] + dense,
            "oracle_dense_fwd_points": [_D, _D] + dense + [_I64P, _I64, _D],
            "oracle_dense_bwd_input": [_D, _D, _D] + dense,
            "oracle_dense_bwd_input_points": [_D, _D] + dense + [_I64P, _I64, _D],
            "oracle_dense_bwd_filter": [_D, _D, _D] + dense,
            "oracle_dense_bwd_filter_taps": [_D, _D] + dense + [_I64P, _I64, _D],
            "oracle_upsample_nearest": [_D, _D, _I64, _I64, _I64, _I64],
            "oracle_upsample_dw_fwd_points": [_D, _D] + six + [_I64, _I64P, _I64, _D],
            "oracle_rgb_to_gray": [_D, _D, _I64, _I64, _I64],
        }
        for name, args in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _INT
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = _INT
        _lib = lib
        return lib


def num_threads() -> int:
    """OpenMP threads the oracle runs on (the CPU-baseline core count)."""
    return int(_load().oracle_num_threads())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_I64P)


def _check(rc: int, name: str) -> None:
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments")


def _dw_shape(x, w, K):
    if x.ndim != 4:
        raise ValueError("x must be NCHW")
    N, C, H, W = x.shape
    if w.shape != (C, K, K):
        raise ValueError(f"w must be (C, K, K) = {(C, K, K)}, got {w.shape}")
    return N, C, H, W


def _filter_size(w) -> int:
    return int(np.asarray(w).shape[-1])


# ------------------------------------------------------------------ depthwise

def dw_fwd(x, w, border: int) -> np.ndarray:
    """y[n,c,i,j] = sum_{a,b} w[c,a,b] * x~[n,c,i+a-r,j+b-r]."""
    x, w = _f64(x), _f64(w)
    K = _filter_size(w)
    N, C, H, W = _dw_shape(x, w, K)
    y = np.empty_like(x)
    _check(_load().oracle_dw_fwd(_p(x), _p(w), _p(y), N, C, H, W, K, border), "dw_fwd")
    return y


def dw_fwd_points(x, w, border: int, idx) -> np.ndarray:
    """Forward outputs at flat NCHW indices ``idx`` only."""
    x, w, idx = _f64(x), _f64(w), _i64(idx)
    K = _filter_size(w)
    N, C, H, W = _dw_shape(x, w, K)
    out = np.empty(idx.size, dtype=np.float64)
    _check(_load().oracle_dw_fwd_points(_p(x), _p(w), N, C, H, W, K, border, _pi(idx),
                                        idx.size, _p(out)), "dw_fwd_points")
    return out


def dw_bwd_input(dy, w, border: int) -> np.ndarray:
    """dx = K^T dy, the transpose of ``dw_fwd`` (scatter form)."""
    dy, w = _f64(dy), _f64(w)
    K = _filter_size(w)
    N, C, H, W = _dw_shape(dy, w, K)
    dx = np.empty_like(dy)
    _check(_load().oracle_dw_bwd_input(_p(dy), _p(w), _p(dx), N, C, H, W, K, border),
           "dw_bwd_input")
    return dx


def dw_bwd_input_points(dy, w, border: int, idx) -> np.ndarray:
    dy, w, idx = _f64(dy), _f64(w), _i64(idx)
    K = _filter_size(w)
    N, C, H, W = _dw_shape(dy, w, K)
    out = np.empty(idx.size, dtype=np.float64)
    _check(_load().oracle_dw_bwd_input_points(_p(dy), _p(w), N, C, H, W, K, border, _pi(idx),
                                              idx.size, _p(out)), "dw_bwd_input_points")
    return out


def dw_bwd_filter(x, dy, K: int, border: int) -> np.ndarray:
    """dw[c,a,b] = sum_{n,i,j} dy[n,c,i,j] * x~[n,c,i+a-r,j+b-r]  -> (C, K, K)."""
    x, dy = _f64(x), _f64(dy)
    N, C, H, W = x.shape
    if dy.shape != x.shape:
        raise ValueError("dy must have the shape of x")
    dw = np.empty((C, K, K), dtype=np.float64)
    _check(_load().oracle_dw_bwd_filter(_p(x), _p(dy), _p(dw), N, C, H, W, K, border),
           "dw_bwd_filter")
    return dw


def dw_bwd_filter_taps(x, dy, K: int, border: int, taps) -> np.ndarray:
    """Filter-gradient entries at flat indices ``c*K*K + a*K + b`` only."""
    x, dy, taps = _f64(x), _f64(dy), _i64(taps)
    N, C, H, W = x.shape
    out = np.empty(taps.size, dtype=np.float64)
    _check(_load().oracle_dw_bwd_filter_taps(_p(x), _p(dy), N, C, H, W, K, border, _pi(taps),
                                             taps.size, _p(out)), "dw_bwd_filter_taps")
    return out


# ---------------------------------------------------------------------- dense

def _dense_shape(x, w):
    if x.ndim != 4 or w.ndim != 4:
        raise ValueError("x must be NHWC and w (Co, K, K, Ci)")
    N, H, W, Ci = x.shape
    Co, K, K2, Ci2 = w.shape
    if K != K2 or Ci2 != Ci:
        raise ValueError("filter shape does not match the input channels")
    return N, H, W, Ci, Co, K


def dense_fwd(x, w, border: int) -> np.ndarray:
    """y[n,i,j,o] = sum_{a,b,c} w[o,a,b,c] * x~[n,i+a-r,j+b-r,c]  (NHWC)."""
    x, w = _f64(x), _f64(w)
    N, H, W, Ci, Co, K = _dense_shape(x, w)
    y = np.empty((N, H, W, Co), dtype=np.float64)
    _check(_load().oracle_dense_fwd(_p(x), _p(w), _p(y), N, H, W, Ci, Co, K, border),
           "dense_fwd")
    return y


def dense_fwd_points(x, w, border: int, idx) -> np.ndarray:
    x, w, idx = _f64(x), _f64(w), _i64(idx)
    N, H, W, Ci, Co, K = _dense_shape(x, w)
    out = np.empty(idx.size, dtype=np.float64)
    _check(_load().oracle_dense_fwd_points(_p(x), _p(w), N, H, W, Ci, Co, K, border, _pi(idx),
                                           idx.size, _p(out)), "dense_fwd_points")
    return out


def dense_bwd_input(dy, w, border: int) -> np.ndarray:
    dy, w = _f64(dy), _f64(w)
    N, H, W, Co = dy.shape
    Co2, K, _, Ci = w.shape
    if Co2 != Co:
        raise ValueError("filter shape does not match dy")
    dx = np.empty((N, H, W, Ci), dtype=np.float64)
    _check(_load().oracle_dense_bwd_input(_p(dy), _p(w), _p(dx), N, H, W, Ci, Co, K, border),
           "dense_bwd_input")
    return dx


def dense_bwd_input_points(dy, w, border: int, idx) -> np.ndarray:
    dy, w, idx = _f64(dy), _f64(w), _i64(idx)
    N, H, W, Co = dy.shape
    Co2, K, _, Ci = w.shape
    out = np.empty(idx.size, dtype=np.float64)
    _check(_load().oracle_dense_bwd_input_points(_p(dy), _p(w), N, H, W, Ci, Co, K, border,
                                                 _pi(idx), idx.size, _p(out)),
           "dense_bwd_input_points")
    return out


def dense_bwd_filter(x, dy, K: int, border: int) -> np.ndarray:
    x, dy = _f64(x), _f64(dy)
    N, H, W, Ci = x.shape
    Co = dy.shape[3]
    dw = np.empty((Co, K, K, Ci), dtype=np.float64)
    _check(_load().oracle_dense_bwd_filter(_p(x), _p(dy), _p(dw), N, H, W, Ci, Co, K, border),
           "dense_bwd_filter")
    return dw


def dense_bwd_filter_taps(x, dy, K: int, border: int, taps) -> np.ndarray:
    x, dy, taps = _f64(x), _f64(dy), _i64(taps)
    N, H, W, Ci = x.shape
    Co = dy.shape[3]
    out = np.empty(taps.size, dtype=np.float64)
    _check(_load().oracle_dense_bwd_filter_taps(_p(x), _p(dy), N, H, W, Ci, Co, K, border,
                                                _pi(taps), taps.size, _p(out)),
           "dense_bwd_filter_taps")
    return out


class use_library:
    """Context manager that points this module at another build of the same C
    source (the mutation tests plant a mistake in a copy and check that the
    pins catch it)."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        self.saved = _load()
        return self._install(ctypes.CDLL(self.path))

    def _install(self, lib):
        global _lib
        for name in ("oracle_dw_fwd", "oracle_dw_fwd_points", "oracle_dw_bwd_input",
                     "oracle_dw_bwd_input_points", "oracle_dw_bwd_filter",
                     "oracle_dw_bwd_filter_taps", "oracle_dense_fwd", "oracle_dense_fwd_points",
                     "oracle_dense_bwd_input", "oracle_dense_bwd_input_points",
                     "oracle_dense_bwd_filter", "oracle_dense_bwd_filter_taps",
                     "oracle_upsample_nearest", "oracle_upsample_dw_fwd_points",
                     "oracle_rgb_to_gray",
                     "oracle_num_threads"):
            src, dst = getattr(self.saved, name), getattr(lib, name)
            dst.argtypes, dst.restype = src.argtypes, src.restype
        with _lock:
            _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


# ----------------------------------------------------------------- upsampling

def upsample_nearest(x, s: int) -> np.ndarray:
    """Nearest-neighbour upsampling by the integer factor s over the last two
    axes (Section 4.2.3): out[..., p, q] = x[..., p // s, q // s]."""
    x = _f64(x)
    *lead, H, W = x.shape
    planes = int(np.prod(lead)) if lead else 1
    y = np.empty((*lead, H * s, W * s), dtype=np.float64)
    _check(_load().oracle_upsample_nearest(_p(x), _p(y), planes, H, W, s), "upsample_nearest")
    return y


def upsample_dw_fwd(x, w, border: int, s: int) -> np.ndarray:
    """The sharpening benchmark (Section 6.6): upsample, then filter."""
    return dw_fwd(upsample_nearest(x, s), w, border)


def upsample_dw_fwd_points(x, w, border: int, s: int, idx) -> np.ndarray:
    """``upsample_dw_fwd`` at flat NCHW indices of the (N, C, H*s, W*s) result."""
    x, w, idx = _f64(x), _f64(w), _i64(idx)
    K = _filter_size(w)
    N, C, H, W = _dw_shape(x, w, K)
    out = np.empty(idx.size, dtype=np.float64)
    _check(_load().oracle_upsample_dw_fwd_points(_p(x), _p(w), N, C, H, W, K, border, s,
                                                 _pi(idx), idx.size, _p(out)),
           "upsample_dw_fwd_points")
    return out


# --------------------------------------------------------- separable filters

def dw_fwd_separable(x, wcol, wrow, border: int) -> np.ndarray:
    """The depthwise filter whose taps are w[c][a][b] = wcol[c][a] * wrow[c][b]
    (the outer product, formed in FP64), applied by the plain definition
    ``dw_fwd``: filtering with a separable filter is the same neighbourhood
    sum as with its full K x K form."""
    wc, wr = _f64(wcol), _f64(wrow)
    if wc.ndim != 2 or wc.shape != wr.shape:
        raise ValueError("wcol and wrow must both be (C, K)")
    return dw_fwd(x, wc[:, :, None] * wr[:, None, :], border)


# ------------------------------------------------------------------ grayscale

def rgb_to_gray(x) -> np.ndarray:
    """Section 4.2.5: gray = 0.299 R + 0.587 G + 0.114 B; x (N, 3, H, W) ->
    (N, 1, H, W)."""
    x = _f64(x)
    if x.ndim != 4 or x.shape[1] != 3:
        raise ValueError("x must be (N, 3, H, W)")
    N, _, H, W = x.shape
    g = np.empty((N, 1, H, W), dtype=np.float64)
    _check(_load().oracle_rgb_to_gray(_p(x), _p(g), N, H, W), "rgb_to_gray")
    return g


def gray_dw_fwd(x, w, border: int) -> np.ndarray:
    """Grayscale conversion, then the filter w (1, K, K) on the gray image."""
    return dw_fwd(rgb_to_gray(x), w, border)
