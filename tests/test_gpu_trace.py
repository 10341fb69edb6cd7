"""GPU check of the log-spaced P(t) / energy trace (the observables of Eq. 3).

In binary64 the chain equals the serial oracle, so every recorded point
(hops, attempts, P, energy) must equal the oracle's running values after the
same number of hops; the recorded attempt counts must pass the log-spaced
thresholds in order; sigma(t) from the windows has the sign of the field.
"""
import math

import numpy as np
import pytest

import oracle

from paper_1407_5026_gb300.sigma import sigma_windows

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


def test_trace_points_follow_the_serial_chain(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.1, E=0.05, seed=5)
    s = B.System([p], precision=B.CG_FP64)
    try:
        obs = s.observables(0)
        Gamma = obs["Gamma"]
        B.cg_set_trace(s.h, first_time=0.05, points_per_decade=10.0, capacity=200)
        s.run(3000, 1024)
        tr = B.cg_read_trace(s.h, 0, 200)
        assert len(tr) >= 10
        ch = oracle.Chain(32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.1, E=0.05, seed=5)
        P0 = ch.counters()["P"]
        E0 = ch.counters()["energy"]
        _, log = ch.run(3000, 1024, log=True)
        m = (log["p"].astype(np.int64) - 1) * 1024 + log["q"]
        att = np.cumsum(m)
        P = P0 + np.cumsum(log["dx"].astype(np.int64))
        # the first point is the state when the trace was set
        assert tr[0]["hops"] == 0 and tr[0]["attempts"] == 0 and tr[0]["P"] == P0
        assert abs(tr[0]["energy"] - E0) <= 1e-9 * max(1.0, abs(E0))
        # the hops that must be recorded: the first hop reaching each threshold,
        # thresholds 0.05 Gamma * ratio^n skipping those a single hop passes
        ratio = math.pow(10.0, 1.0 / 10.0)
        want, nxt = [], 0.05 * Gamma
        for h in range(1, 3001):
            if len(want) + 1 >= 200:
                break
            if att[h - 1] >= nxt:
                want.append(h)
                while nxt <= att[h - 1]:
                    nxt = max(nxt * ratio, nxt + 1.0)
        assert [int(x) for x in tr["hops"][1:]] == want
        for k in range(1, len(tr)):
            h = int(tr[k]["hops"])
            assert tr[k]["attempts"] == att[h - 1]
            assert tr[k]["P"] == P[h - 1]
        t, sig = sigma_windows(tr, 32 * 32, 0.05)
        assert np.all(np.diff(t) > 0)
        assert sig[len(sig) // 2:].mean() > 0      # current along the field
    finally:
        s.close()
