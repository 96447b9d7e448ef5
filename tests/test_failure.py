"""Failure detection without a GPU fault: every device wait in the library
is bounded; when one runs out the kernel records GIGA_ERR_TIMEOUT in a device
error word and returns, and the host reads it through
giga_check_device_error.  The self-test entry point makes such a wait run out
on purpose (a barrier nothing completes, given up after 2 s), then the test
checks the reported status and that the context still computes correctly.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_TOL, normwise, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def giga():
    import paper_2504_01266_gb300 as g
    from paper_2504_01266_gb300 import build
    build.build()
    return g


def test_bounded_wait_reports_timeout_and_device_stays_usable(giga):
    from paper_2504_01266_gb300 import _lib
    st = torch.cuda.current_stream().cuda_stream
    assert _lib.giga_check_device_error(st) == _lib.GIGA_OK
    t0 = time.time()
    assert _lib.giga_selftest_bounded_wait(st) == _lib.GIGA_OK
    assert _lib.giga_check_device_error(st) == _lib.GIGA_ERR_TIMEOUT
    waited = time.time() - t0
    assert 1.5 < waited < 60, waited
    assert _lib.giga_check_device_error(st) == _lib.GIGA_OK  # read once, then cleared
    # the context is intact: a TMA-staged forward still matches the oracle
    gen = torch.Generator().manual_seed(17)
    x = torch.rand((1, 2, 96, 256), generator=gen)
    w = torch.randn((2, 5, 5), generator=gen) * 0.1
    y = giga.conv2d_fwd(x.cuda(), w.cuda(), "clamp")
    torch.cuda.synchronize()
    assert _lib.giga_check_device_error(st) == _lib.GIGA_OK
    ref = oracle.dw_fwd(x.numpy(), w.numpy(), oracle.CLAMP)
    assert normwise(to_np(y), ref) <= FP32_TOL
    assert np.isfinite(to_np(y)).all()
