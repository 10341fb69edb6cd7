"""GPU tower sampler (guide table + thresholds) against the oracle's binary
search over the integer cumulative weights (hop vector by tower sampling,
section "Hopping conduction in the Coulomb glass").

Every threshold and its neighbours, every guide-bucket edge and its
neighbours, the extremes of the 32-bit range and 2^20 random words must map
to the same vector index (or to the null proposal) on both sides.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

GUIDE_BITS = 12

CASES = [dict(L=16, xi=1.0, r_max=4), dict(L=64, xi=1.0, r_max=6),
         dict(L=128, xi=1.0, r_max=8), dict(L=256, xi=1.5, r_max=10),
         dict(L=64, xi=3.0, r_max=20)]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def _words(C):
    C = C.astype(np.int64)
    pts = [0, 1, 2, (1 << 32) - 2, (1 << 32) - 1]
    for c in C:
        pts += [c - 2, c - 1, c, c + 1]
    for b in range(1 << GUIDE_BITS):
        lo = b << (32 - GUIDE_BITS)
        pts += [lo - 1, lo, lo + 1]
    pts = np.array([p for p in pts if 0 <= p < (1 << 32)], dtype=np.uint64)
    rnd = np.random.default_rng(7).integers(0, 1 << 32, size=1 << 20, dtype=np.uint64)
    return np.concatenate([pts, rnd]).astype(np.uint32)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{c['L']}_xi{c['xi']}_r{c['r_max']}")
def test_tower_matches_oracle(B, case):
    p = dict(nu=0.5, W=1.0, T=0.05, E=0.0, seed=1, **case)
    s = B.System([p], precision=B.CG_FP64)
    try:
        ch = oracle.Chain(case["L"], nu=0.5, W=1.0, xi=case["xi"], r_max=case["r_max"],
                          T=0.05, E=0.0, seed=1)
        _, _, Wi, _ = ch.vectors()
        C = np.cumsum(Wi.astype(np.uint64))
        x1 = _words(C)
        got = B.cg_debug_tower(s.h, 0, x1)
        want = ch.tower(x1)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (x1[bad[:5]], got[bad[:5]], want[bad[:5]])
        # the null region is exactly [C_{V-1}, 2^32)
        assert np.all((want == -1) == (x1.astype(np.uint64) >= C[-1]))
    finally:
        s.close()
