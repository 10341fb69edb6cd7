"""GPU checks of the stochastic time increment (mixed PR algorithm, step 3c,
reading R13: each executed hop adds max(0, (m + sqrt(m) z) / Gamma), z from
Box-Muller on the hop's own Philox block).

The GPU deviates equal the oracle's bit for bit; in binary64 the stochastic
clock of a run (single CTA and thread-block cluster) equals the serial
oracle's; trace points carry the time (attempts / Gamma by default, the
stochastic clock otherwise); group I/O carries it; in binary32 the clock
tracks attempts / Gamma within its standard deviation.
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


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _oracle_for(p, mode=1):
    ch = oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"], T=p["T"],
                      E=p["E"], seed=p["seed"], replica=p.get("replica", 0))
    ch.set_time_mode(mode)
    return ch


def test_gpu_deviates_equal_the_oracle(B):
    rng = np.random.default_rng(4)
    n = 20000
    seeds = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    seeds[:8] = [0, 1, 2, 5, 1 << 40, (1 << 64) - 1, 12345, 1 << 32]
    reps = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    hops = rng.integers(0, 1 << 45, n, dtype=np.uint64)
    hops[:8] = [0, 1, 2, (1 << 32) - 1, 1 << 32, (1 << 40) + 3, 7, 999]
    got = B.cg_debug_gauss(seeds, reps, hops)
    want = np.array([oracle.gauss(int(s), int(r), int(h)) for s, r, h in zip(seeds, reps, hops)])
    bad = np.nonzero(_bits(got) != _bits(want))[0]
    assert bad.size == 0, (seeds[bad[:3]], hops[bad[:3]], got[bad[:3]], want[bad[:3]])


@pytest.mark.parametrize("L,cluster", [(32, 0), (48, 2), (64, 4)])
def test_binary64_stochastic_clock_equals_the_oracle(B, L, cluster):
    p = dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=21, replica=2)
    s = B.System([p], precision=B.CG_FP64, time_mode=B.CG_TIME_GAUSSIAN, cluster_size=cluster)
    try:
        for hops, M in ((1500, 1024), (700, 333)):
            s.run(hops, M)
        c = s.state(0)[3]
        ch = _oracle_for(p)
        ch.run(1500, 1024)
        ch.run(700, 333)
        oc = ch.counters()
        assert c["hops"] == oc["hops"] and c["attempts"] == oc["attempts"]
        assert c["time"] == oc["time"]
        obs = s.observables(0)
        assert obs["time"] == oc["time"]
        assert abs(obs["time"] - oc["attempts"] / obs["Gamma"]) < 6 * math.sqrt(oc["attempts"]) / obs["Gamma"]
    finally:
        s.close()


def test_trace_points_carry_the_time(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.1, E=0.05, seed=5)
    for mode in (B.CG_TIME_DETERMINISTIC, B.CG_TIME_GAUSSIAN):
        s = B.System([p], precision=B.CG_FP64, time_mode=mode)
        try:
            Gamma = s.observables(0)["Gamma"]
            B.cg_set_trace(s.h, first_time=0.05, points_per_decade=10.0, capacity=200)
            s.run(3000, 1024)
            tr = B.cg_read_trace(s.h, 0, 200)
            assert len(tr) >= 10
            if mode == B.CG_TIME_DETERMINISTIC:
                for pt in tr[1:]:
                    assert pt["time"] == float(pt["attempts"]) / Gamma
            else:
                # the clock at the hop each point was recorded at
                ch = _oracle_for(p)
                t_at = {}
                for h in range(1, 3001):
                    ch.run(1, 1024)
                    t_at[h] = ch.counters()["time"]
                for pt in tr[1:]:
                    assert pt["time"] == t_at[int(pt["hops"])]
            t, sig = sigma_windows(tr, 32 * 32, 0.05)
            assert np.all(np.diff(t) > 0) and np.isfinite(sig).all()
        finally:
            s.close()


def test_group_io_carries_the_time(B):
    reps = [dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=k, replica=k)
            for k in range(4)]
    a = B.System(reps, precision=B.CG_FP64, time_mode=B.CG_TIME_GAUSSIAN)
    b = B.System(reps, precision=B.CG_FP64, time_mode=B.CG_TIME_GAUSSIAN)
    try:
        a.run(400, 512)
        occ, eps, cnt = a.read_group(0)
        assert np.all(cnt["time"] > 0)
        b.write_group(0, occ=occ, eps=eps, counters=cnt)
        a.run(300, 512)
        b.run(300, 512)
        for k in range(4):
            assert a.state(k)[3]["time"] == b.state(k)[3]["time"]
    finally:
        a.close()
        b.close()


def test_binary32_stochastic_clock_tracks_attempts(B):
    reps = [dict(L=64, nu=0.5, W=2.0, xi=1.0, r_max=6, T=0.02, E=0.005, seed=s, replica=s)
            for s in range(16)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=1024, time_mode=B.CG_TIME_GAUSSIAN)
    try:
        s.run(3000, 2048)
        for k in range(16):
            o = s.observables(k)
            att = o["attempts"]
            assert o["time"] > 0
            assert abs(o["time"] - att / o["Gamma"]) < 6 * math.sqrt(att) / o["Gamma"]
    finally:
        s.close()
