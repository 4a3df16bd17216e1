"""The measurement probes the bench reports its FP64 and L2 fractions against
(dbfft_fp64_fma_rate, dbfft_l2_copy_rate): each returns a finite rate in the
range a GB300-class GPU can have, and a second call agrees with the first to
a few percent (best of several timed launches)."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def test_fp64_fma_rate_is_plausible_and_repeatable():
    dbfft = _dbfft()
    a, b = dbfft.fp64_fma_rate(), dbfft.fp64_fma_rate()
    assert math.isfinite(a) and 0.05 < a < 200.0  # TFLOP/s
    assert abs(a - b) <= 0.1 * max(a, b)


def test_l2_copy_rate_is_plausible_and_repeatable():
    dbfft = _dbfft()
    a, b = dbfft.l2_copy_rate(), dbfft.l2_copy_rate()
    assert math.isfinite(a) and 500.0 < a < 200000.0  # GB/s
    assert abs(a - b) <= 0.15 * max(a, b)
