"""GPU checks of the random-site chain on thread-block clusters (one replica
over 2, 4 or 8 CTAs, each owning a contiguous range of sites' eps).

Binary64, so the cluster form's hops are the serial chain's bit for bit:
every logged hop, the final occupation, eps and the counters equal the
oracle's on forced clusters (including CTAs that own no site) and a batch
on 4-CTA clusters equals the single-CTA kernel's; boxes past one CTA's
shared memory (L = 176, and L = 256 with a 34 GB coupling matrix) take a
cluster by themselves, two splits of them give the same chain, and eps
stays equal to its definition.  A hop that can never end returns
CG_ETIMEOUT with the state intact.
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


def _oracle_for(p):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"], T=p["T"],
                        E=p["E"], seed=p["seed"], replica=p.get("replica", 0),
                        random_sites=True)


FIELDS = ("i", "j", "q", "p", "round", "dx", "dy", "k", "l", "dx2", "dy2")


def _check_same(s, idx, ch, log=None, olog=None):
    if log is not None:
        for f in FIELDS:
            np.testing.assert_array_equal(log[f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log["dE"]), _bits(olog["dE"]))
    n, eps, _, cnt = s.state(idx)
    on, oeps, _ = ch.state()
    np.testing.assert_array_equal(n, on)
    np.testing.assert_array_equal(_bits(eps), _bits(oeps))
    oc = ch.counters()
    for f in ("rounds", "hops", "attempts", "P"):
        assert cnt[f] == oc[f], f
    assert abs(cnt["energy"] - oc["energy"]) <= 1e-9 * max(1.0, abs(oc["energy"]))


def _p(B, **kw):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.1, E=0.01, seed=8, replica=1,
             sites=B.CG_SITES_RANDOM)
    p.update(kw)
    return p


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("L,r_max,xi,T,E,M,threads", [
    (16, 3, 1.0, 0.1, 0.01, 1024, 256),
    # N = 324: on 8 CTAs each owns 64 sites, CTA 5 four, CTAs 6 and 7 none
    (18, 4, 0.7, 0.2, 0.05, 333, 512),
    (32, 6, 1.0, 0.05, 0.0, 4096, 1024),
], ids=lambda v: str(v))
def test_random_cluster_trajectory_bit_exact(B, L, r_max, xi, T, E, M, threads, cluster):
    p = _p(B, L=L, r_max=r_max, xi=xi, T=T, E=E, seed=13, replica=2)
    s = B.System([p], precision=B.CG_FP64, cluster_size=cluster, block_threads=threads)
    try:
        sh = B.cg_group_shape(s.h, 0)
        assert sh["cluster"] == cluster and sh["threads"] == threads
        ch = _oracle_for(p)
        _check_same(s, 0, ch)
        rc, log = s.run_logged(1000, M)
        assert rc == B.CG_OK
        _, olog = ch.run(1000, M, log=True)
        _check_same(s, 0, ch, log[0], olog)
        # a second launch continues the chain from the stored state
        assert s.run(300, M) == B.CG_OK
        assert ch.run(300, M)[0] == oracle.ORC_OK
        _check_same(s, 0, ch)
    finally:
        s.close()


def test_random_cluster_batch_equals_single_cta(B):
    # four replicas of L = 96 (N = 9216) on 4-CTA clusters and on one CTA
    # each: the same chains, hop for hop
    reps = [_p(B, L=96, r_max=5, T=0.05, seed=40 + k, replica=k) for k in range(4)]
    a = B.System(reps, precision=B.CG_FP64)
    b = B.System(reps, precision=B.CG_FP64, cluster_size=4)
    try:
        assert B.cg_group_shape(a.h, 0)["cluster"] == 1
        assert B.cg_group_shape(b.h, 0)["cluster"] == 4
        ra, la = a.run_logged(2000, 2048)
        rb, lb = b.run_logged(2000, 2048)
        assert ra == rb == B.CG_OK
        for k in range(4):
            for f in FIELDS:
                np.testing.assert_array_equal(la[k][f], lb[k][f], err_msg=f)
            np.testing.assert_array_equal(_bits(la[k]["dE"]), _bits(lb[k]["dE"]))
            na, ea, _, ca = a.state(k)
            nb, eb, _, cb = b.state(k)
            np.testing.assert_array_equal(na, nb)
            np.testing.assert_array_equal(_bits(ea), _bits(eb))
            for f in ("rounds", "hops", "attempts", "energy"):
                assert ca[f] == cb[f], f
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("L,auto,other", [(176, 2, 4), (256, 4, 8)])
def test_random_sites_past_one_cta_on_clusters(B, L, auto, other):
    # L = 176 (eps of N = 30976 sites, 242 KiB) and L = 256 (N = 65536, a
    # 34 GB coupling matrix) outgrow one CTA, so the handle puts each replica
    # on a cluster by itself.  The handle's split and a finer one hold
    # different site ranges per CTA and give the same chain; every logged
    # hop moves one electron from an occupied site to an empty partner
    # within r_max; after the hops the running eps equals eps rebuilt from
    # its definition within the rounding of the updates.  (The serial oracle
    # needs minutes to build a box this large; the cluster kernel is checked
    # against it hop for hop on the smaller boxes above.)
    p = _p(B, L=L, r_max=6, T=0.05, E=0.005, seed=2, replica=0)
    R = float(p["r_max"])
    a = B.System([p], precision=B.CG_FP64, torch_memory=False)
    try:
        assert B.cg_group_shape(a.h, 0)["cluster"] == auto
        n0 = a.state(0)[0]
        ra, la = a.run_logged(2000, 4096)
        assert ra == B.CG_OK
        na, ea, _, ca = a.state(0)
        x, y = B.cg_site_positions(a.h, 0)
        occ = n0.astype(np.int8).copy()
        h = L / 2.0
        for e in la[0]:
            i, j = int(e["i"]), int(e["j"])
            assert occ[i] == 1 and occ[j] == 0
            dx = (x[j] - x[i] + h) % L - h
            dy = (y[j] - y[i] + h) % L - h
            assert dx * dx + dy * dy <= R * R + 1e-9
            occ[i], occ[j] = 0, 1
        np.testing.assert_array_equal(occ, na)
        B.cg_refresh(a.h)
        assert np.max(np.abs(ea - a.state(0)[1])) < 1e-9
    finally:
        a.close()
    b = B.System([p], precision=B.CG_FP64, torch_memory=False, cluster_size=other)
    try:
        assert B.cg_group_shape(b.h, 0)["cluster"] == other
        rb, lb = b.run_logged(2000, 4096)
        assert rb == B.CG_OK
        for f in FIELDS:
            np.testing.assert_array_equal(la[0][f], lb[0][f], err_msg=f)
        np.testing.assert_array_equal(_bits(la[0]["dE"]), _bits(lb[0]["dE"]))
        nb, eb, _, cb = b.state(0)
        np.testing.assert_array_equal(na, nb)
        np.testing.assert_array_equal(_bits(ea), _bits(eb))
        for f in ("rounds", "hops", "attempts", "energy"):
            assert ca[f] == cb[f], f
    finally:
        b.close()


@pytest.mark.parametrize("cluster", [0, 2, 4])
def test_random_hop_time_limit_returns_timeout(B, cluster):
    # at T = 1e-12 a hop accepts only when dH <= ~1e-9 (exp(-dH/T) is 0
    # beyond that), so the chain descends to a state that no single hop
    # lowers, and the next hop never ends: the wall-clock limit (rank 0's on
    # a cluster) stops it, the launch stores a valid state and the counters
    # hold complete failed rounds only; max_rounds_per_hop bounds the wait
    # a second time
    p = _p(B, L=18, r_max=3, T=1e-12, E=0.0, seed=3, replica=0)
    s = B.System([p], precision=B.CG_FP64, cluster_size=cluster, hop_timeout_ms=200,
                 max_rounds_per_hop=1 << 22)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] == max(cluster, 1)
        with pytest.raises(B.CgError) as ei:
            s.run(20000, 1024)
        assert ei.value.code == B.CG_ETIMEOUT
        n1, e1, _, c1 = s.state(0)
        assert 0 < c1["hops"] < 20000
        ch = _oracle_for(p)
        assert ch.run(c1["hops"], 1024)[0] == oracle.ORC_OK
        on, oe, _ = ch.state()
        oc = ch.counters()
        np.testing.assert_array_equal(n1, on)
        np.testing.assert_array_equal(_bits(e1), _bits(oe))
        assert c1["rounds"] > oc["rounds"]
        assert c1["attempts"] - oc["attempts"] == 1024 * (c1["rounds"] - oc["rounds"])
    finally:
        s.close()


def test_random_cluster_autotune_keeps_the_chain(B):
    # the autotuner times cluster sizes 1, 2, 4 and 8 for random sites on a
    # snapshot it restores
    p = _p(B, L=48, r_max=4, T=0.1, seed=12)
    s = B.System([p], precision=B.CG_FP64)
    try:
        B.cg_autotune(s.h, 64)
        sh = B.cg_group_shape(s.h, 0)
        assert sh["cluster"] in (1, 2, 4, 8)
        rc, log = s.run_logged(400, 512)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(400, 512, log=True)
        _check_same(s, 0, ch, log[0], olog)
    finally:
        s.close()
