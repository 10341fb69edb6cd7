"""GPU checks of the batched form: replicas of several L in one handle,
concurrent launches per L, CUDA-graph replay, and the launch-shape autotuner.

* A captured-graph handle and a plain handle over the same replicas give
  bit-identical states (the graph replays the same launches).
* In binary64 every replica of a mixed-L batch still equals its serial chain.
* The autotuner restores every replica's state bit for bit after its trials,
  picks shapes that fit, and reuses a JSON cache.
"""
import json
import os

import numpy as np
import pytest

import oracle

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


def _mixed(R, T=0.03, seed0=0):
    sizes = [32, 48, 64, 96]
    return [dict(L=sizes[k % 4], nu=0.5, W=1.0, xi=1.0, r_max=6, T=T, E=0.01,
                 seed=seed0 + k, replica=seed0 + k) for k in range(R)]


def test_graph_replay_equals_plain_launches(B):
    reps = _mixed(24)
    a = B.System(reps, precision=B.CG_FP32, refresh_every=256,
                 refresh_kind=B.CG_REFRESH_BF16X2, use_graph=0)
    b = B.System(reps, precision=B.CG_FP32, refresh_every=256,
                 refresh_kind=B.CG_REFRESH_BF16X2, use_graph=1)
    try:
        assert B.cg_num_groups(a.h) == 4
        for hops in (300, 300, 212, 300):      # repeated shapes replay cached graphs
            a.run(hops, 2048)
            b.run(hops, 2048)
        for k in range(len(reps)):
            sa, sb = a.state(k), b.state(k)
            np.testing.assert_array_equal(sa[0], sb[0])
            np.testing.assert_array_equal(_bits(sa[1]), _bits(sb[1]))
            assert sa[3] == sb[3]
            assert a.observables(k)["refreshes"] == b.observables(k)["refreshes"] == 4
    finally:
        a.close()
        b.close()


def test_mixed_binary64_batch_with_graph_is_bit_exact(B):
    reps = _mixed(8, T=0.05, seed0=40)
    s = B.System(reps, precision=B.CG_FP64, use_graph=1)
    try:
        for _ in range(3):
            s.run(400, 1024)
        for k in (0, 1, 2, 3, 7):
            p = reps[k]
            ch = oracle.Chain(p["L"], nu=0.5, W=1.0, xi=1.0, r_max=6, T=p["T"], E=0.01,
                              seed=p["seed"], replica=p["replica"])
            for _ in range(3):
                ch.run(400, 1024)
            n, eps, _, c = s.state(k)
            on, oeps, _ = ch.state()
            np.testing.assert_array_equal(n, on)
            np.testing.assert_array_equal(_bits(eps), _bits(oeps))
            assert c["attempts"] == ch.counters()["attempts"]
    finally:
        s.close()


def test_autotune_restores_state_and_caches(B, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("CG_TUNE_CACHE", str(cache))
    reps = _mixed(8, T=0.05, seed0=80)
    s = B.System(reps, precision=B.CG_FP64)
    try:
        s.run(200, 1024)
        before = [s.state(k) for k in range(len(reps))]
        B.cg_autotune(s.h, 64)
        for k in range(len(reps)):
            after = s.state(k)
            np.testing.assert_array_equal(before[k][0], after[0])
            np.testing.assert_array_equal(_bits(before[k][1]), _bits(after[1]))
            assert before[k][3] == after[3]
        shapes = [B.cg_group_shape(s.h, g) for g in range(B.cg_num_groups(s.h))]
        for sh in shapes:
            # single-CTA groups need one thread per base column (L/2); the
            # cluster kernel one per column (L)
            assert sh["threads"] in (256, 384, 512, 1024) and 2 * sh["threads"] >= sh["L"]
            assert sh["M"] in (1024, 4096, 16384, 65536)
            assert sh["cluster"] in (1, 2, 4, 8)
            assert sh["cluster"] == 1 or (sh["threads"] >= sh["L"] and sh["L"] % (2 * sh["cluster"]) == 0)
        data = json.loads(cache.read_text())
        assert len(data) == len(shapes)
        # M = 0 runs each group with its tuned M; binary64 still matches the
        # serial chain with that M
        s.run(300, 0)
        k = 0
        M0 = next(sh["M"] for sh in shapes if sh["L"] == reps[k]["L"])
        p = reps[k]
        ch = oracle.Chain(p["L"], nu=0.5, W=1.0, xi=1.0, r_max=6, T=p["T"], E=0.01,
                          seed=p["seed"], replica=p["replica"])
        ch.run(200, 1024)
        ch.run(300, M0)
        np.testing.assert_array_equal(_bits(s.state(k)[1]), _bits(ch.state()[1]))
    finally:
        s.close()
    # a new handle reuses the cached shapes without trials
    s2 = B.System(reps, precision=B.CG_FP64)
    try:
        B.cg_autotune(s2.h, 64)
        shapes2 = [B.cg_group_shape(s2.h, g) for g in range(B.cg_num_groups(s2.h))]
        assert shapes2 == shapes
    finally:
        s2.close()
