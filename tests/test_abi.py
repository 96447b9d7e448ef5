"""CPU checks of the C ABI boundary: the library loads without a GPU, exports
every symbol include/giga.h declares, and rejects bad arguments before any
CUDA call (only host-side paths run here)."""
import ctypes
import json
import os
import re

import pytest

from paper_2504_01266_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_01266_gb300 import build
    build.build()
    return _lib.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "giga.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(giga_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert header_functions() == sorted(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def dw(N=1, C=3, H=16, W=16, K=3, border=0, dtype=0):
    return _lib.desc(N, C, C, H, W, K, C, border, dtype, _lib.GIGA_LAYOUT_NCHW)


@pytest.mark.parametrize("field,value,status", [
    ("K", 4, _lib.GIGA_ERR_INVALID_ARG),
    ("K", 0, _lib.GIGA_ERR_INVALID_ARG),
    ("K", 33, _lib.GIGA_ERR_INVALID_ARG),
    ("border", 5, _lib.GIGA_ERR_INVALID_ARG),
    ("dtype", 9, _lib.GIGA_ERR_INVALID_ARG),
    ("H", -1, _lib.GIGA_ERR_INVALID_ARG),
    ("reserved", 1, _lib.GIGA_ERR_INVALID_ARG),
    ("layout", _lib.GIGA_LAYOUT_NHWC, _lib.GIGA_ERR_UNSUPPORTED),
])
def test_bad_descriptor(lib, field, value, status):
    d = dw()
    setattr(d, field, value)
    fake = 0x10000  # never dereferenced: validation fails first
    assert _lib.giga_conv2d_fwd(d, fake, fake, fake * 2, None, 0, None) == status
    assert _lib.last_error_detail() != ""


def test_null_and_misaligned_pointers(lib):
    d = dw()
    assert _lib.giga_conv2d_fwd(d, None, 0x10000, 0x20000, None, 0, None) == \
        _lib.GIGA_ERR_INVALID_ARG
    assert _lib.giga_conv2d_fwd(d, 0x10001, 0x10000, 0x20000, None, 0, None) == \
        _lib.GIGA_ERR_MISALIGNED


def test_aliasing_rejected(lib):
    d = dw()
    assert _lib.giga_conv2d_fwd(d, 0x10000, 0x90000, 0x10040, None, 0, None) == \
        _lib.GIGA_ERR_INVALID_ARG
    assert "alias" in _lib.last_error_detail()


def test_workspace_sizes(lib):
    d = dw(N=2, C=3, H=100, W=300, K=7)
    assert _lib.giga_conv2d_workspace_size(d, _lib.GIGA_OP_FWD) == 0
    assert _lib.giga_conv2d_workspace_size(d, _lib.GIGA_OP_BWD_INPUT) == 0
    n = _lib.giga_conv2d_workspace_size(d, _lib.GIGA_OP_BWD_FILTER)
    tiles = ((300 + 127) // 128) * ((100 + 63) // 64)
    assert n >= 2 * 3 * tiles * 49 * 4 and n % 256 == 0


def test_workspace_errors(lib):
    d = dw(N=1, C=1, H=64, W=128, K=3)
    need = _lib.giga_conv2d_workspace_size(d, _lib.GIGA_OP_BWD_FILTER)
    a = 0x100000
    assert _lib.giga_conv2d_bwd_filter(d, a, a * 2, a * 3, None, 0, None) == _lib.GIGA_ERR_WORKSPACE
    assert _lib.giga_conv2d_bwd_filter(d, a, a * 2, a * 3, a * 4, need - 1, None) == \
        _lib.GIGA_ERR_WORKSPACE
    assert _lib.giga_conv2d_bwd_filter(d, a, a * 2, a * 3, a * 4 + 16, need, None) == \
        _lib.GIGA_ERR_WORKSPACE


def test_filter_gradient_k_limit(lib):
    d = dw(K=17)
    a = 0x100000
    assert _lib.giga_conv2d_bwd_filter(d, a, a * 2, a * 3, a * 4, 1 << 30, None) == \
        _lib.GIGA_ERR_UNSUPPORTED


def test_status_strings(lib):
    for s in range(7):
        assert _lib.status_string(s)


def test_autotune_cache_roundtrip_and_corruption(lib, tmp_path):
    path = str(tmp_path / "cache.json")
    _lib.giga_autotune_clear()
    assert _lib.giga_autotune_save(path) == _lib.GIGA_OK
    data = json.load(open(path))
    assert data["giga_autotune"] == 1 and data["entries"] == {}
    data["entries"]["0:0:3:0:20"] = 1
    json.dump(data, open(path, "w"))
    assert _lib.giga_autotune_load(path) == _lib.GIGA_OK
    d = dw(N=1, C=1, H=1024, W=1024, K=3)  # 2^20 elements -> size class 20
    assert _lib.giga_autotune_choice(d, _lib.GIGA_OP_FWD) == 1
    # a corrupt file is ignored: the call reports it and the cache is kept
    open(path, "w").write("{not json")
    assert _lib.giga_autotune_load(path) == _lib.GIGA_ERR_INVALID_ARG
    assert _lib.giga_autotune_choice(d, _lib.GIGA_OP_FWD) == 1
    _lib.giga_autotune_clear()
    assert _lib.giga_autotune_choice(d, _lib.GIGA_OP_FWD) == 0
    with pytest.raises(_lib.GigaError):
        _lib.giga_autotune_set_mode(7)


def test_autotune_set_choice(lib):
    _lib.giga_autotune_clear()
    mode = _lib.giga_autotune_get_mode()
    _lib.giga_autotune_set_mode(1)
    try:
        d = dw(N=2, C=3, H=256, W=512, K=15)
        fused = _lib.GIGA_OP_BWD_INPUT | _lib.GIGA_OP_BWD_FILTER
        assert _lib.giga_autotune_set_choice(d, fused, 6) == _lib.GIGA_OK
        assert _lib.giga_autotune_set_choice(d, fused, 7) == _lib.GIGA_ERR_INVALID_ARG
        assert _lib.giga_autotune_set_choice(d, fused, 5) == _lib.GIGA_OK
        assert _lib.giga_autotune_choice(d, fused) == 5
        assert _lib.giga_autotune_choice(d, _lib.GIGA_OP_FWD) == 0  # other ops untouched
        assert _lib.giga_autotune_set_choice(d, _lib.GIGA_OP_FWD, 7) == _lib.GIGA_OK
        assert _lib.giga_autotune_set_choice(d, _lib.GIGA_OP_FWD, 8) == _lib.GIGA_ERR_INVALID_ARG
        assert _lib.giga_autotune_set_choice(d, _lib.GIGA_OP_BWD_FILTER, 5) == \
            _lib.GIGA_ERR_INVALID_ARG
        assert _lib.giga_autotune_set_choice(d, 3, 0) == _lib.GIGA_ERR_INVALID_ARG
        assert _lib.giga_autotune_set_choice(d, _lib.GIGA_OP_FWD, -1) == _lib.GIGA_ERR_INVALID_ARG
    finally:
        _lib.giga_autotune_clear()
        _lib.giga_autotune_set_mode(mode)


def test_empty_problem_launches_nothing(lib):
    d = dw(N=0)
    _lib.giga_launch_count_reset()
    assert _lib.giga_conv2d_fwd(d, None, None, None, None, 0, None) == _lib.GIGA_OK
    assert _lib.giga_launch_count() == 0
