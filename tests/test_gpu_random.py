"""GPU checks of the random-site Coulomb glass (reading R16) against the
serial oracle.

Binary64, so every logged hop (sites, label, round, dH bit for bit), the
final occupation, eps bit for bit and the counters equal the oracle's:
for powers of two and other even L, with and without a field, with the
guide records in shared memory and (lists of 256 pairs or more) in global
memory, one replica
and a batch that mixes random-site and lattice replicas (graph replay
included).  A refresh rebuilds eps from its definition bit for bit; every
CTA size and the autotuner keep the chain; the lattice-only calls refuse.
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
                        random_sites=bool(p.get("sites", 0)))


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


@pytest.mark.parametrize("L,r_max,xi,T,E,M", [
    (8, 2, 1.0, 0.3, 0.02, 256),
    (16, 3, 1.0, 0.1, 0.0, 1024),
    (18, 4, 0.7, 0.2, 0.05, 333),
    (32, 6, 1.0, 0.05, 0.01, 4096),
    # lists of about 314 pairs: the guide records stay in global memory (the
    # shared-memory copy takes lists below 256 pairs)
    (32, 10, 1.5, 0.05, 0.01, 4096),
], ids=lambda v: str(v))
def test_binary64_random_site_trajectory_bit_exact(B, L, r_max, xi, T, E, M):
    p = dict(L=L, nu=0.5, W=1.0, xi=xi, r_max=r_max, T=T, E=E, seed=13, replica=2,
             sites=B.CG_SITES_RANDOM)
    s = B.System([p], precision=B.CG_FP64)
    try:
        ch = _oracle_for(p)
        # the set-up state: eps from its definition, bit for bit
        _check_same(s, 0, ch)
        rc, log = s.run_logged(1200, M)
        assert rc == B.CG_OK
        _, olog = ch.run(1200, M, log=True)
        _check_same(s, 0, ch, log[0], olog)
        assert (log[0]["dx"] == 0).all() and (log[0]["k"] == 0xFFFFFFFF).all()
        obs = s.observables(0)
        assert obs["Gamma"] == ch.Gamma == L * L * ch.Zmax
        assert obs["time"] == ch.counters()["attempts"] / ch.Gamma
        # a refresh rebuilds eps from scratch in the definition's order
        B.cg_refresh(s.h)
        np.testing.assert_array_equal(_bits(s.state(0)[1]), _bits(ch.eps_scratch()))
    finally:
        s.close()


def test_mixed_batch_of_random_and_lattice_replicas(B):
    base = dict(nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.1, E=0.02)
    reps = [dict(base, L=16, seed=3 + k, replica=k, sites=B.CG_SITES_RANDOM) for k in range(3)]
    reps += [dict(base, L=16, seed=9, replica=7), dict(base, L=12, seed=4, replica=1,
                                                      sites=B.CG_SITES_RANDOM)]
    s = B.System(reps, precision=B.CG_FP64, use_graph=1)
    try:
        for _ in range(2):
            assert s.run(300, 512) == B.CG_OK
        for idx, p in enumerate(reps):
            ch = _oracle_for(p)
            assert ch.run(600, 512)[0] == oracle.ORC_OK
            _check_same(s, idx, ch)
    finally:
        s.close()


def test_random_site_state_round_trip(B):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.1, E=0.0, seed=21, replica=0,
             sites=B.CG_SITES_RANDOM)
    s = B.System([p], precision=B.CG_FP64)
    try:
        assert s.run(200, 1024) == B.CG_OK
        n, eps, phi, cnt = s.state(0)
        # writing the occupation alone rebuilds eps from scratch
        B.cg_write_state(s.h, 0, n, None, phi)
        ch = _oracle_for(p)
        assert ch.run(200, 1024)[0] == oracle.ORC_OK
        np.testing.assert_array_equal(s.state(0)[0], ch.state()[0])
        np.testing.assert_array_equal(_bits(s.state(0)[1]), _bits(ch.eps_scratch()))
    finally:
        s.close()


def _random_p(B, **kw):
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.1, E=0.01, seed=8, replica=1,
             sites=B.CG_SITES_RANDOM)
    p.update(kw)
    return p


@pytest.mark.parametrize("threads", [256, 384, 512])
def test_random_site_cta_sizes_bit_exact(B, threads):
    # every CTA size evaluates the labels in its own chunks; the hops are
    # the serial chain's
    p = _random_p(B)
    s = B.System([p], precision=B.CG_FP64, block_threads=threads)
    try:
        assert B.cg_group_shape(s.h, 0)["threads"] == threads
        rc, log = s.run_logged(600, 700)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(600, 700, log=True)
        _check_same(s, 0, ch, log[0], olog)
    finally:
        s.close()


def test_random_site_autotune_keeps_the_chain(B):
    # the autotuner's trial launches run on a snapshot that is restored
    p = _random_p(B, seed=12)
    s = B.System([p], precision=B.CG_FP64)
    try:
        B.cg_autotune(s.h, 64)
        assert B.cg_group_shape(s.h, 0)["threads"] in (256, 384, 512, 1024)
        rc, log = s.run_logged(400, 512)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(400, 512, log=True)
        _check_same(s, 0, ch, log[0], olog)
    finally:
        s.close()


def test_random_site_handle_refuses_lattice_only_calls(B):
    s = B.System([_random_p(B)], precision=B.CG_FP64)
    try:
        with pytest.raises(B.CgError, match="constant-acceptance"):
            B.cg_set_toy_acceptance(s.h, 0.5)
        with pytest.raises(B.CgError, match="partner lists"):
            B.cg_debug_tower(s.h, 0, [1, 2, 3])
        assert s.run(50, 256) == B.CG_OK
    finally:
        s.close()


def test_site_positions_equal_the_oracle(B):
    p = _random_p(B, L=12, seed=3, replica=5)
    s = B.System([p, dict(p, sites=0)], precision=B.CG_FP64)
    try:
        x, y = B.cg_site_positions(s.h, 0)
        ox, oy = _oracle_for(p).positions()
        np.testing.assert_array_equal(_bits(x), _bits(ox))
        np.testing.assert_array_equal(_bits(y), _bits(oy))
        with pytest.raises(B.CgError, match="lattice"):
            B.cg_site_positions(s.h, 1)
    finally:
        s.close()
