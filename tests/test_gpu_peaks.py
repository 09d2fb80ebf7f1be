"""The pipe-peak measurement helpers (needs a GPU): finite, positive rates, FP32 above FP64."""
import math

import pytest

from paper_1901_07643_gb300 import binding

pytestmark = pytest.mark.gpu


def test_fma_and_dmma_peaks_are_plausible():
    f32, f64 = binding.pipe_peaks()
    mma64 = binding.dmma_peak()
    for v in (f32, f64, mma64):
        assert math.isfinite(v) and v > 0
    assert f32 > f64
    # a warp instruction is 512 flops; any rate above 100 PFLOP/s would mean the chains were dropped
    assert mma64 < 1e5
