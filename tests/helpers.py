"""Shared helpers of the GPU parity tests (metrics and tolerances).

Tolerances, with the reading of the error metric used throughout:
  * normwise relative error  max|out - ref| / max|ref|  per output tensor (an
    elementwise ratio is meaningless where outputs cross zero);
  * FP32 storage: <= 1e-5 against the FP64 oracle on the same inputs;
  * BF16 storage, FP32 accumulation:
      - against the FP64 oracle on the BF16-rounded inputs (kernel error only):
        <= 2^-8, one rounding of the output to BF16 (2^-9 relative) with margin;
      - against the FP64 oracle on the original FP32 inputs (end to end):
        <= 1e-2.
"""
import numpy as np
import torch

FP32_TOL = 1e-5
BF16_KERNEL_TOL = 2.0 ** -8
BF16_E2E_TOL = 1e-2
U32 = 2.0 ** -24          # unit roundoff of FP32
NORMWISE_MIN_ELEMS = 16   # fewer outputs than this have no meaningful norm


def gamma(n: int) -> float:
    """Classic bound on the relative error of an n-term FP32 sum of products."""
    return n * U32 / (1.0 - n * U32)


def assert_fp32(out, ref, mag, n_terms: int, what=""):
    """FP32 result against the FP64 oracle.

    * every element: |out - ref| <= gamma(n_terms) * mag, where mag is the same
      operator applied to the magnitudes |w|, |x| (the sum of |terms|) -- the
      rigorous forward-error bound of FP32 accumulation, valid even where the
      exact value cancels to almost nothing;
    * the normwise relative error max|out - ref| / max|ref| <= 1e-5 whenever
      the output has at least NORMWISE_MIN_ELEMS elements.
    """
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mag = np.asarray(mag, dtype=np.float64)
    assert not np.isnan(out).any(), f"{what}: NaN in output (unwritten element?)"
    bound = gamma(n_terms) * mag + 1e-30
    bad = np.abs(out - ref) > bound
    assert not bad.any(), f"{what}: {int(bad.sum())} elements beyond the FP32 bound"
    if out.size >= NORMWISE_MIN_ELEMS:
        err = normwise(out, ref)
        assert err <= FP32_TOL, f"{what}: normwise {err:.3e}"


def normwise(out, ref) -> float:
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max() if ref.size else 0.0
    if scale == 0.0:
        return float(np.abs(out).max()) if out.size else 0.0
    return float(np.abs(out - ref).max() / scale)


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).numpy()


def poison_like(t: torch.Tensor) -> torch.Tensor:
    """Output buffer filled with NaN so unwritten elements show up."""
    return torch.full_like(t, float("nan"))
