"""GPU checks of two-electron hops (the multi-electron hops the paper names
as an extension of its GPU code; reading R15) against the serial oracle.

In binary64 every logged hop (both electrons of a pair, dH bit for bit), the
final state and the counters equal the oracle's, for powers of two and other
even L, with and without a field; the pair kernel with T_p = 0 runs the
single-hop chain; in binary32 (refreshed) eps stays within 1e-4 of its
definition, the hop log replays to the device state, and the chain follows
the binary64 one hop for hop until a near tie.
"""
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


def _oracle_for(p, pair_frac, pair_rmax):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"], T=p["T"],
                        E=p["E"], seed=p["seed"], replica=p.get("replica", 0),
                        pair_frac=pair_frac, pair_rmax=pair_rmax)


FIELDS = ("i", "j", "q", "p", "round", "dx", "dy", "k", "l", "dx2", "dy2")


@pytest.mark.parametrize("L,r_max,T,E,pf,R,M", [
    (16, 4, 0.3, 0.02, 0.3, 3, 256),
    (16, 3, 0.1, 0.0, 0.5, 2, 1024),
    (18, 4, 0.3, 0.05, 0.2, 4, 333),
    (32, 6, 0.2, 0.01, 0.3, 5, 512),
], ids=lambda v: str(v))
def test_binary64_pair_trajectory_bit_exact(B, L, r_max, T, E, pf, R, M):
    p = dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=r_max, T=T, E=E, seed=11, replica=3)
    s = B.System([p], precision=B.CG_FP64, pair_frac=pf, pair_rmax=R)
    try:
        rc, log = s.run_logged(1500, M)
        assert rc == B.CG_OK
        ch = _oracle_for(p, pf, R)
        _, olog = ch.run(1500, M, log=True)
        g = log[0]
        for f in FIELDS:
            np.testing.assert_array_equal(g[f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(g["dE"]), _bits(olog["dE"]))
        assert (g["k"] != 0xFFFFFFFF).sum() >= 10        # pairs were executed
        n, eps, _, cnt = s.state(0)
        on, oeps, _ = ch.state()
        np.testing.assert_array_equal(n, on)
        np.testing.assert_array_equal(_bits(eps), _bits(oeps))
        oc = ch.counters()
        for f in ("rounds", "hops", "attempts", "P"):
            assert cnt[f] == oc[f], f
        assert abs(cnt["energy"] - oc["energy"]) <= 1e-9 * max(1.0, abs(oc["energy"]))
        obs = s.observables(0)
        assert obs["Gamma"] == ch.Gamma
        assert obs["time"] == oc["attempts"] / ch.Gamma
    finally:
        s.close()


def test_pair_kernel_without_pair_labels_is_the_single_hop_chain(B):
    # pair_frac > 0 selects the pair kernel; floor(p2 2^32) = 0 draws no pair
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.01, seed=5)
    s = B.System([p], precision=B.CG_FP64, pair_frac=1e-12, pair_rmax=3)
    try:
        rc, log = s.run_logged(1200, 256)
        assert rc == B.CG_OK
        ch = _oracle_for(p, 0.0, 0)
        _, olog = ch.run(1200, 256, log=True)
        for f in FIELDS:
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log[0]["dE"]), _bits(olog["dE"]))
        np.testing.assert_array_equal(_bits(s.state(0)[1]), _bits(ch.state()[1]))
    finally:
        s.close()


def test_binary64_pair_batch_and_graph(B):
    reps = [dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.3, E=0.02, seed=s, replica=s)
            for s in range(6)]
    s = B.System(reps, precision=B.CG_FP64, pair_frac=0.25, pair_rmax=3, use_graph=1)
    try:
        for hops, M in ((300, 512), (300, 512), (200, 128)):
            assert s.run(hops, M) == B.CG_OK
        for k, p in enumerate(reps):
            ch = _oracle_for(p, 0.25, 3)
            for hops, M in ((300, 512), (300, 512), (200, 128)):
                ch.run(hops, M)
            n, eps, _, cnt = s.state(k)
            on, oeps, _ = ch.state()
            np.testing.assert_array_equal(n, on)
            np.testing.assert_array_equal(_bits(eps), _bits(oeps))
            assert cnt["P"] == ch.counters()["P"]
    finally:
        s.close()


def test_binary32_pair_runs(B):
    L, R = 32, 4
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.2, E=0.01, seed=s, replica=s)
            for s in range(12)]
    s32 = B.System(reps, precision=B.CG_FP32, refresh_every=256, pair_frac=0.2, pair_rmax=R)
    s64 = B.System(reps, precision=B.CG_FP64, pair_frac=0.2, pair_rmax=R)
    try:
        rc, log32 = s32.run_logged(2000, 512)
        assert rc == B.CG_OK
        rc, log64 = s64.run_logged(2000, 512)
        assert rc == B.CG_OK
        same_prefix = []
        for k, p in enumerate(reps):
            n, eps, phi, cnt = s32.state(k)
            o = s32.observables(k)
            assert o["refreshes"] >= 7 and o["max_eps_err_last_refresh"] <= 1e-4
            ch = _oracle_for(p, 0.2, R)
            ch.set_state(n, phi)
            assert np.abs(eps - ch.state()[1]).max() <= 1e-4
            # the log replays to the device state and the dipole
            g = log32[k]
            n0 = _oracle_for(p, 0.2, R).state()[0].astype(np.int64)
            pair = g["k"] != 0xFFFFFFFF
            for e, pr in zip(g, pair):
                assert n0[e["i"]] == 1 and n0[e["j"]] == 0
                n0[e["i"]], n0[e["j"]] = 0, 1
                if pr:
                    assert n0[e["k"]] == 1 and n0[e["l"]] == 0
                    n0[e["k"]], n0[e["l"]] = 0, 1
            np.testing.assert_array_equal(n0, n)
            P0 = _oracle_for(p, 0.2, R).counters()["P"]
            assert cnt["P"] - P0 == int(g["dx"].sum() + g["dx2"].sum())
            # binary32 follows binary64 hop for hop until a near tie
            h64 = log64[k]
            diff = np.nonzero((g["i"] != h64["i"]) | (g["q"] != h64["q"]) |
                              (g["k"] != h64["k"]))[0]
            same_prefix.append(diff[0] if diff.size else len(g))
        assert (log32["k"] != 0xFFFFFFFF).sum() >= 100
        assert np.median(same_prefix) >= 200, same_prefix
    finally:
        s32.close()
        s64.close()


def test_binary64_pair_stochastic_clock_bit_exact(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.3, E=0.02, seed=8, replica=1)
    s = B.System([p], precision=B.CG_FP64, pair_frac=0.3, pair_rmax=3,
                 time_mode=B.CG_TIME_GAUSSIAN)
    try:
        rc, log = s.run_logged(1200, 256)
        assert rc == B.CG_OK
        ch = _oracle_for(p, 0.3, 3)
        ch.set_time_mode(1)
        _, olog = ch.run(1200, 256, log=True)
        for f in FIELDS:
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
        assert (log[0]["k"] != 0xFFFFFFFF).sum() >= 10
        cnt = s.state(0)[3]
        assert cnt["time"] == ch.counters()["time"]
        assert s.observables(0)["time"] == ch.counters()["time"]
    finally:
        s.close()


@pytest.mark.parametrize("L,cluster", [(32, 2), (48, 4), (64, 8)])
def test_binary64_pair_cluster_bit_exact(B, L, cluster):
    # the pair data crosses the cluster: four energies through distributed
    # shared memory, the second electron in its own exchange slot
    p = dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=5, T=0.3, E=0.02, seed=13, replica=2)
    s = B.System([p], precision=B.CG_FP64, pair_frac=0.3, pair_rmax=4, cluster_size=cluster)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] == cluster
        rc, log = s.run_logged(1200, 512)
        assert rc == B.CG_OK
        ch = _oracle_for(p, 0.3, 4)
        _, olog = ch.run(1200, 512, log=True)
        for f in FIELDS:
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log[0]["dE"]), _bits(olog["dE"]))
        assert (log[0]["k"] != 0xFFFFFFFF).sum() >= 10
        n, eps, _, cnt = s.state(0)
        on, oeps, _ = ch.state()
        np.testing.assert_array_equal(n, on)
        np.testing.assert_array_equal(_bits(eps), _bits(oeps))
        assert cnt["P"] == ch.counters()["P"]
    finally:
        s.close()


def test_binary32_pairs_beyond_one_cta(B):
    # L=256 in binary32 needs a 2-CTA cluster
    reps = [dict(L=256, nu=0.5, W=1.0, xi=1.5, r_max=10, T=0.05, E=0.005, seed=s, replica=s)
            for s in range(2)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=2048, pair_frac=0.2, pair_rmax=4)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] >= 2
        rc, log = s.run_logged(4500, 4096)
        assert rc == B.CG_OK
        assert (log["k"] != 0xFFFFFFFF).sum() >= 5
        for k in range(2):
            o = s.observables(k)
            assert o["refreshes"] == 2 and o["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()


def _cubic_oracle(p, pf, R, mode=0):
    ch = oracle.Chain(p["L"], dim=3, nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                      T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0),
                      pair_frac=pf, pair_rmax=R)
    ch.set_time_mode(mode)
    return ch


@pytest.mark.parametrize("L,R,pf,M,cluster", [(8, 2, 0.5, 256, 0), (6, 2, 0.6, 128, 0),
                                              (10, 3, 0.5, 300, 0), (16, 2, 0.5, 512, 2),
                                              (16, 2, 0.5, 512, 4)])
def test_binary64_cubic_pair_trajectory_bit_exact(B, L, R, pf, M, cluster):
    p = dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=2, T=0.5, E=0.02, seed=12, replica=1, dim=3)
    s = B.System([p], precision=B.CG_FP64, pair_frac=pf, pair_rmax=R, cluster_size=cluster)
    try:
        if cluster:
            assert B.cg_group_shape(s.h, 0)["cluster"] == cluster
        rc, log = s.run_logged(1500, M)
        assert rc == B.CG_OK
        ch = _cubic_oracle(p, pf, R)
        _, olog = ch.run(1500, M, log=True)
        for f in FIELDS:
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log[0]["dE"]), _bits(olog["dE"]))
        assert (log[0]["k"] != 0xFFFFFFFF).sum() >= 10
        n, eps, _, cnt = s.state(0)
        on, oeps, _ = ch.state()
        np.testing.assert_array_equal(n, on)
        np.testing.assert_array_equal(_bits(eps), _bits(oeps))
        assert cnt["P"] == ch.counters()["P"]
    finally:
        s.close()


def test_cubic_pair_stochastic_clock_and_binary32(B):
    p = dict(L=8, nu=0.5, W=1.0, xi=1.0, r_max=2, T=0.5, E=0.02, seed=12, replica=1, dim=3)
    s = B.System([p], precision=B.CG_FP64, pair_frac=0.5, pair_rmax=2,
                 time_mode=B.CG_TIME_GAUSSIAN)
    try:
        s.run(1200, 256)
        ch = _cubic_oracle(p, 0.5, 2, mode=1)
        ch.run(1200, 256)
        assert s.state(0)[3]["time"] == ch.counters()["time"]
    finally:
        s.close()
    reps = [dict(p, seed=k, replica=k, L=16) for k in range(8)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=256, pair_frac=0.4, pair_rmax=2)
    try:
        rc, log = s.run_logged(1500, 512)
        assert rc == B.CG_OK
        assert (log["k"] != 0xFFFFFFFF).sum() >= 20
        for k in (0, 7):
            n, eps, phi, _ = s.state(k)
            ch = _cubic_oracle(reps[k], 0.4, 2)
            ch.set_state(n, phi)
            assert np.abs(eps - ch.state()[1]).max() <= 1e-4
    finally:
        s.close()
