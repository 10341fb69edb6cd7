"""GPU checks of the library's microbenchmarks (the measured peaks and
barrier costs bench.py divides by): every kind returns a finite positive
value in a plausible range for one GPU of this class, the same order of
magnitude on a second call; the barrier kinds come out between a few
nanoseconds and a hundred microseconds.
"""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


RANGES = {
    0: (1e12, 1e15),     # shared-memory RMW bytes/s (32-bit words), all SMs
    1: (1e10, 1e14),     # binary64 adds/s
    2: (1e12, 1e15),     # shared-memory RMW bytes/s (64-bit words)
    3: (1e10, 1e14),     # Philox-4x32-10 blocks/s
    4: (1e-9, 1e-4),     # seconds per cluster barrier, 2 CTAs
    5: (1e-9, 1e-4),     # 4 CTAs
    6: (1e-9, 1e-4),     # 8 CTAs
    7: (1e-9, 1e-4),     # seconds per CTA barrier, 1024 threads
}


@pytest.mark.parametrize("kind", sorted(RANGES))
def test_microbench_values_are_plausible(B, kind):
    lo, hi = RANGES[kind]
    a = B.cg_microbench(kind, 0)
    b = B.cg_microbench(kind, 0)
    for v in (a, b):
        assert math.isfinite(v) and lo < v < hi, (kind, v)
    assert 0.5 < a / b < 2.0, (kind, a, b)
