"""GPU parity of the binary64 path against the CPU oracle (bit-exact).

Everything is called through the C ABI (ctypes binding).  The PR kernel and
the serial oracle consume the same Philox streams, so the parallel rejection
chain must reproduce the serial chain exactly (parallel rejection section:
the two algorithms are mathematically equivalent); in binary64 with matching
operation order the equality is bit for bit: every hop (i, j, label q, rounds
p, round counter, dH), the final occupation, eps, phi and the counters.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads

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


def _oracle_for(p):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0))


def _assert_state_equal(sysm, k, ch):
    n, eps, phi, cnt = sysm.state(k)
    on, oeps, ophi = ch.state()
    np.testing.assert_array_equal(n, on)
    np.testing.assert_array_equal(_bits(phi), _bits(ophi))
    bad = np.nonzero(_bits(eps) != _bits(oeps))[0]
    assert len(bad) == 0, f"eps differs at {len(bad)} sites, first {bad[:5]}"
    oc = ch.counters()
    for f in ("rounds", "hops", "attempts", "P"):
        assert cnt[f] == oc[f], (f, cnt[f], oc[f])
    # the running energy starts from Eq. 1 evaluated through eps, so it agrees
    # to rounding, not bit for bit
    assert abs(cnt["energy"] - oc["energy"]) <= 1e-9 * max(1.0, abs(oc["energy"]))


def _assert_log_equal(log, olog):
    for f in ("i", "j", "q", "p", "round", "dx", "dy"):
        if not np.array_equal(log[f], olog[f]):
            h = int(np.nonzero(log[f] != olog[f])[0][0])
            raise AssertionError(f"hop {h}: field {f} gpu={log[h]} oracle={olog[h]}")
    np.testing.assert_array_equal(_bits(log["dE"]), _bits(olog["dE"]))


def test_philox_gpu_equals_oracle(B):
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = B.cg_debug_philox(ctr, key)
    for t in range(n):
        np.testing.assert_array_equal(out[t], oracle.philox(ctr[t], key[t]))


def test_acceptance_exp_gpu_equals_oracle(B):
    rng = np.random.default_rng(1)
    x = np.concatenate([-23.0 * rng.random(20000), -np.logspace(-15, 1.36, 3000),
                        [0.0, -0.0, -23.0, -22.999999999, -23.0000001, -1e-300,
                         -math.log(2), -0.5 * math.log(2)]])
    got = B.cg_debug_exp(x)
    want = np.array([oracle.cg_exp(v) for v in x])
    bad = np.nonzero(_bits(got) != _bits(want))[0]
    assert len(bad) == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])


@pytest.mark.parametrize("L,W,r_max,seed", [(16, 1.0, 4, 0), (48, 1.0, 6, 3), (64, 1.0, 6, 5),
                                            (128, 2.0, 8, 0), (6, 1.0, 2, 9)])
def test_initial_state_bit_exact(B, L, W, r_max, seed):
    p = dict(L=L, nu=0.5, W=W, xi=1.0, r_max=r_max, T=0.05, E=0.01, seed=seed)
    sysm = B.System([p], precision=B.CG_FP64)
    try:
        _assert_state_equal(sysm, 0, _oracle_for(p))
    finally:
        sysm.close()


def test_l16_trajectory_bit_exact_every_hop(B):
    wl = workloads.l16_fp64()
    p = wl.replicas[0].as_dict()
    sysm = B.System([p], precision=B.CG_FP64)
    try:
        rc, log = sysm.run_logged(wl.hops, wl.M)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        orc, olog = ch.run(wl.hops, wl.M, log=True)
        assert orc == oracle.ORC_OK
        _assert_log_equal(log[0], olog)
        _assert_state_equal(sysm, 0, ch)
        cnt = sysm.state(0)[3]
        assert cnt["evaluated"] >= cnt["attempts"]
    finally:
        sysm.close()


@pytest.mark.parametrize("T", workloads.L64_TEMPERATURES)
@pytest.mark.parametrize("seed", [0, 5])
def test_l64_prefix_bit_exact(B, T, seed):
    wl = workloads.l64_fp64(T=T, seed=seed, hops=3000)
    p = wl.replicas[0].as_dict()
    sysm = B.System([p], precision=B.CG_FP64)
    try:
        rc, log = sysm.run_logged(wl.hops, wl.M)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(wl.hops, wl.M, log=True)
        _assert_log_equal(log[0], olog)
        _assert_state_equal(sysm, 0, ch)
    finally:
        sysm.close()


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_launch_shape_does_not_change_the_chain(B, threads):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.03, E=0.02, seed=11)
    sysm = B.System([p], precision=B.CG_FP64, block_threads=threads)
    try:
        sysm.run(1500, 777)
        ch = _oracle_for(p)
        ch.run(1500, 777)
        _assert_state_equal(sysm, 0, ch)
    finally:
        sysm.close()


def test_split_runs_and_changing_M_equal_the_serial_chain(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.08, E=0.05, seed=21)
    sysm = B.System([p], precision=B.CG_FP64)
    ch = _oracle_for(p)
    try:
        for hops, M in [(100, 1), (250, 64), (1, 4096), (400, 300), (7, 1)]:
            sysm.run(hops, M)
            ch.run(hops, M)
            _assert_state_equal(sysm, 0, ch)
    finally:
        sysm.close()


def test_mixed_sizes_in_one_batch(B):
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=r, T=T, E=0.01, seed=s, replica=s)
            for s, (L, r, T) in enumerate([(16, 4, 0.05), (48, 6, 0.03), (32, 6, 0.1),
                                           (64, 6, 0.02), (16, 3, 0.2), (96, 6, 0.03)])]
    sysm = B.System(reps, precision=B.CG_FP64)
    try:
        rc, log = sysm.run_logged(600, 512)
        assert rc == B.CG_OK
        for k, p in enumerate(reps):
            ch = _oracle_for(p)
            _, olog = ch.run(600, 512, log=True)
            _assert_log_equal(log[k], olog)
            _assert_state_equal(sysm, k, ch)
    finally:
        sysm.close()


def test_write_state_then_run_matches_oracle(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=2)
    n = workloads.random_occupation(256, 128, seed=5)
    phi = workloads.random_phi(256, 1.0, seed=6)
    sysm = B.System([p], precision=B.CG_FP64)
    ch = _oracle_for(p)
    try:
        B.cg_write_state(sysm.h, 0, n, phi=phi)
        ch.set_state(n, phi)
        _assert_state_equal(sysm, 0, ch)
        sysm.run(500, 128)
        ch.run(500, 128)
        _assert_state_equal(sysm, 0, ch)
        # resume from a saved state in a fresh handle (checkpoint / restart)
        n1, e1, p1, c1 = sysm.state(0)
        other = B.System([p], precision=B.CG_FP64)
        try:
            B.cg_write_state(other.h, 0, n1, eps=e1, phi=p1, counters=c1)
            other.run(300, 128)
            ch.run(300, 128)
            _assert_state_equal(other, 0, ch)
        finally:
            other.close()
    finally:
        sysm.close()


def test_write_state_rejects_wrong_electron_count(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=2)
    sysm = B.System([p], precision=B.CG_FP64)
    try:
        n = np.zeros(256, np.uint8)
        n[:100] = 1
        with pytest.raises(B.CgError) as ei:
            B.cg_write_state(sysm.h, 0, n)
        assert ei.value.code == B.CG_ESTATE
    finally:
        sysm.close()


def test_constant_acceptance_mode_matches_oracle(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=3)
    for A0, M in [(0.01, 256), (3e-4, 4096), (0.5, 3)]:
        sysm = B.System([p], precision=B.CG_FP64)
        try:
            B.cg_set_toy_acceptance(sysm.h, A0)
            rc, log = sysm.run_logged(400, M)
            ch = _oracle_for(p)
            ch.set_toy(A0)
            _, olog = ch.run(400, M, log=True)
            for f in ("q", "p", "round", "i"):
                np.testing.assert_array_equal(log[0][f], olog[f])
            c = sysm.state(0)[3]
            assert c["attempts"] == ch.counters()["attempts"]
        finally:
            sysm.close()


def test_max_rounds_returns_stuck_with_valid_state(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=3)
    sysm = B.System([p], precision=B.CG_FP64, max_rounds_per_hop=5)
    try:
        n0, e0, _, c0 = sysm.state(0)
        B.cg_set_toy_acceptance(sysm.h, 0.0)      # no label ever accepts
        rc = sysm.run(1, 64)
        assert rc == B.CG_ESTUCK
        n1, e1, _, c1 = sysm.state(0)
        np.testing.assert_array_equal(n0, n1)
        np.testing.assert_array_equal(_bits(e0), _bits(e1))
        assert c1["rounds"] == c0["rounds"] + 5
        assert c1["attempts"] == c0["attempts"] + 5 * 64
        assert c1["hops"] == c0["hops"]
        # the handle stays usable
        B.cg_set_toy_acceptance(sysm.h, -1.0)
        assert sysm.run(10, 64) == B.CG_OK
    finally:
        sysm.close()


def test_hop_time_limit_returns_timeout(B):
    # a hop that never ends (no label accepts, unbounded rounds) stops at the
    # device wall-clock limit instead of running on
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=3)
    sysm = B.System([p], precision=B.CG_FP64, hop_timeout_ms=200)
    try:
        B.cg_set_toy_acceptance(sysm.h, 0.0)
        with pytest.raises(B.CgError) as ei:
            sysm.run(1, 1024)
        assert ei.value.code == B.CG_ETIMEOUT
        B.cg_set_toy_acceptance(sysm.h, -1.0)
        assert sysm.run(5, 64) == B.CG_OK
    finally:
        sysm.close()


def test_malloc_and_workspace_modes_agree(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=8)
    a = B.System([p], precision=B.CG_FP64, torch_memory=True)
    b = B.System([p], precision=B.CG_FP64, torch_memory=False)
    try:
        a.run(700, 333)
        b.run(700, 333)
        sa, sb = a.state(0), b.state(0)
        np.testing.assert_array_equal(sa[0], sb[0])
        np.testing.assert_array_equal(_bits(sa[1]), _bits(sb[1]))
        assert sa[3] == sb[3]
    finally:
        a.close()
        b.close()
