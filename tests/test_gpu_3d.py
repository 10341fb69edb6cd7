"""GPU checks of the cubic lattice (cg_replica_desc.dim = 3; the
three-dimensional extension of the lattice model named in the paper's
conclusions) against the serial oracle on the L x L x L torus.

In binary64 the initial state, every logged hop and the final state are
bit-identical to the oracle's for powers of two and other even L, with and
without a field; the tower sampler on cubic tables equals the oracle's; a
batch that mixes square and cubic replicas keeps each chain exact; the
stochastic clock of step 3c is exact in 3D too; in binary32 (refreshed in
binary64) eps stays within 1e-4 of its definition, and at L = 32 on one CTA
(L fixed at compile time) eps tracks its definition without a refresh, the
logged hops replay on the occupations and the first hops equal the binary64
serial chain's; the split-BF16 tensor-core
refresh on cubic tables (N = L^3 a multiple of 128) gives eps within 5e-5 of
its definition, alone and inside runs; on thread-block clusters (eps split
by z-planes, 1/r of the update indexed by r^2) binary64 stays bit-exact and
binary32 lattices beyond one CTA (L = 40, 48) refresh within 1e-4; the 64^3
lattice runs in binary32 on 8-CTA clusters, its eps within 1e-4 of the
definition, its hops valid.
"""
import numpy as np
import pytest

import oracle
from tests import physics_ref as ref

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
    ch = oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"], T=p["T"],
                      E=p["E"], seed=p["seed"], replica=p.get("replica", 0),
                      dim=p.get("dim", 2))
    return ch


def _cubic(**kw):
    p = dict(nu=0.5, W=1.0, xi=1.0, T=0.1, E=0.01, seed=5, replica=0, dim=3)
    p.update(kw)
    return p


def _assert_same(B, s, k, p, ch, log=None, olog=None):
    if log is not None:
        for f in ("i", "j", "q", "p", "round", "dx", "dy"):
            np.testing.assert_array_equal(log[f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log["dE"]), _bits(olog["dE"]))
    n, eps, phi, cnt = s.state(k)
    on, oeps, ophi = ch.state()
    np.testing.assert_array_equal(n, on)
    np.testing.assert_array_equal(_bits(phi), _bits(ophi))
    np.testing.assert_array_equal(_bits(eps), _bits(oeps))
    oc = ch.counters()
    for f in ("rounds", "hops", "attempts", "P"):
        assert cnt[f] == oc[f], f
    assert abs(cnt["energy"] - oc["energy"]) <= 1e-9 * max(1.0, abs(oc["energy"]))


@pytest.mark.parametrize("L,r_max", [(8, 2), (6, 2), (10, 3), (16, 3)])
def test_initial_state_bit_exact(B, L, r_max):
    p = _cubic(L=L, r_max=r_max)
    s = B.System([p], precision=B.CG_FP64)
    try:
        assert B.cg_num_sites(s.h, 0) == L ** 3
        _assert_same(B, s, 0, p, _oracle_for(p))
    finally:
        s.close()


@pytest.mark.parametrize("L,r_max,T,E,M", [(8, 2, 0.1, 0.01, 256), (6, 2, 0.05, 0.0, 64),
                                           (10, 3, 0.2, 0.05, 500), (16, 3, 0.05, 0.02, 1024)])
def test_cubic_trajectory_bit_exact(B, L, r_max, T, E, M):
    p = _cubic(L=L, r_max=r_max, T=T, E=E)
    s = B.System([p], precision=B.CG_FP64)
    try:
        rc, log = s.run_logged(1500, M)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(1500, M, log=True)
        _assert_same(B, s, 0, p, ch, log[0], olog)
    finally:
        s.close()


def test_tower_on_cubic_tables(B):
    p = _cubic(L=16, r_max=4, xi=1.5)
    s = B.System([p], precision=B.CG_FP64)
    try:
        ch = _oracle_for(p)
        _, _, Wi, _ = ch.vectors()
        C = np.cumsum(Wi.astype(np.uint64)).astype(np.int64)
        x1 = np.concatenate([C - 1, C, C + 1,
                             np.random.default_rng(2).integers(0, 1 << 32, 200000)])
        x1 = x1[(x1 >= 0) & (x1 < (1 << 32))].astype(np.uint32)
        np.testing.assert_array_equal(B.cg_debug_tower(s.h, 0, x1), ch.tower(x1))
    finally:
        s.close()


def test_batch_mixing_square_and_cubic_replicas(B):
    reps = [dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.01, seed=1, replica=0),
            _cubic(L=8, r_max=2, seed=2, replica=1),
            dict(L=8, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.05, E=0.01, seed=3, replica=2),
            _cubic(L=8, r_max=2, seed=4, replica=3, T=0.3)]
    s = B.System(reps, precision=B.CG_FP64, use_graph=1)
    try:
        assert B.cg_num_groups(s.h) == 3          # (2D, 8), (2D, 16), (3D, 8)
        rc, log = s.run_logged(700, 300)
        assert rc == B.CG_OK
        for k, p in enumerate(reps):
            ch = _oracle_for(p)
            _, olog = ch.run(700, 300, log=True)
            _assert_same(B, s, k, p, ch, log[k], olog)
    finally:
        s.close()


def test_cubic_stochastic_clock_bit_exact(B):
    p = _cubic(L=8, r_max=2)
    s = B.System([p], precision=B.CG_FP64, time_mode=B.CG_TIME_GAUSSIAN)
    try:
        s.run(1000, 256)
        ch = _oracle_for(p)
        ch.set_time_mode(1)
        ch.run(1000, 256)
        assert s.state(0)[3]["time"] == ch.counters()["time"]
    finally:
        s.close()


def test_cubic_binary32_with_binary64_refresh(B):
    reps = [_cubic(L=16, r_max=3, T=0.05, seed=s, replica=s) for s in range(6)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=256, refresh_kind=B.CG_REFRESH_FP64)
    try:
        s.run(2000, 512)
        for k in range(6):
            o = s.observables(k)
            assert o["refreshes"] >= 7 and o["max_eps_err_last_refresh"] <= 1e-4
            n, eps, phi, _ = s.state(k)
            ch = _oracle_for(reps[k])
            ch.set_state(n, phi)
            assert np.max(np.abs(eps - ch.state()[1])) <= 1e-4
    finally:
        s.close()


@pytest.mark.parametrize("threads", [1024, 512, 256])
def test_cubic_binary32_l32_one_cta(B, threads):
    # binary32 at L = 32 on one CTA (the instance with L fixed at compile
    # time): with no refresh, eps after 1500 hops stays within 1e-4 of its
    # definition (every site of the octant update gets its 1/r terms); the
    # logged hops move an electron from an occupied site to an empty one
    # within r_max and reproduce the final occupation; the first hops equal
    # the binary64 serial chain's (no near tie among them on these seeds)
    L, r_max = 32, 3
    reps = [_cubic(L=L, r_max=r_max, T=0.05, seed=s, replica=s) for s in range(3)]
    s = B.System(reps, precision=B.CG_FP32, cluster_size=1, block_threads=threads)
    try:
        sh = B.cg_group_shape(s.h, 0)
        assert sh["cluster"] == 1 and sh["threads"] == threads
        occ0 = [s.state(k)[0].astype(np.int8).copy() for k in range(3)]
        rc, log = s.run_logged(1500, 1024)
        assert rc == B.CG_OK
        for k in range(3):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - ref.site_energies_fft3(n, phi, 0.5, L)).max() <= 1e-4
            occ = occ0[k]
            for e in log[k]:
                i, j = int(e["i"]), int(e["j"])
                assert occ[i] == 1 and occ[j] == 0
                d = [((j // L**a) % L - (i // L**a) % L + L // 2) % L - L // 2
                     for a in range(3)]
                assert 0 < d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= r_max * r_max
                occ[i], occ[j] = 0, 1
            np.testing.assert_array_equal(occ, n)
        ch = _oracle_for(reps[0])
        _, olog = ch.run(30, 1024, log=True)
        for f in ("i", "j", "q", "p", "round"):
            np.testing.assert_array_equal(log[0][f][:30], olog[f], err_msg=f)
    finally:
        s.close()


@pytest.mark.parametrize("L,R", [(8, 9), (16, 40), (24, 17), (32, 152)])
def test_cubic_tensor_core_refresh_matches_definition(B, L, R):
    # D = G (2n - 1) with G built from the (L/2+1)^3 folded table on the fly
    reps = [_cubic(L=L, r_max=3, T=0.05, seed=s, replica=s) for s in range(R)]
    s = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_BF16X2)
    try:
        s.run(40, 256)
        B.cg_refresh(s.h)
        worst = 0.0
        for k in sorted({0, 1, R // 2, R - 1}):
            n, eps, phi, _ = s.state(k)
            exact = ref.site_energies_fft3(n, phi, 0.5, L)
            worst = max(worst, float(np.abs(eps - exact).max()))
            obs = s.observables(k)
            assert obs["refreshes"] == 1 and obs["max_eps_err_last_refresh"] <= 1e-4
        assert worst <= 5e-5, worst
    finally:
        s.close()


def test_cubic_tensor_core_refresh_in_runs(B):
    # 16 cubic replicas refreshed on the tensor cores inside runs
    reps = [_cubic(L=16, r_max=3, T=0.03, seed=s, replica=s) for s in range(16)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=256,
                 refresh_kind=B.CG_REFRESH_BF16X2)
    try:
        s.run(4 * 256 + 50, 1024)
        for k in (0, 7, 15):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - ref.site_energies_fft3(n, phi, 0.5, 16)).max() <= 1e-4
            o = s.observables(k)
            assert o["refreshes"] == 4 and o["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()


@pytest.mark.parametrize("L,cluster,E", [(16, 2, 0.01), (16, 4, 0.0), (16, 8, 0.03),
                                         (24, 2, 0.02), (24, 8, 0.01)])
def test_cubic_cluster_trajectory_bit_exact(B, L, cluster, E):
    p = _cubic(L=L, r_max=3, T=0.1, E=E, seed=6, replica=1)
    s = B.System([p], precision=B.CG_FP64, cluster_size=cluster)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] == cluster
        rc, log = s.run_logged(1500, 512)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(1500, 512, log=True)
        _assert_same(B, s, 0, p, ch, log[0], olog)
    finally:
        s.close()


def test_cubic_cluster_stochastic_clock(B):
    p = _cubic(L=16, r_max=2, seed=3)
    s = B.System([p], precision=B.CG_FP64, cluster_size=4, time_mode=B.CG_TIME_GAUSSIAN)
    try:
        s.run(800, 256)
        ch = _oracle_for(p)
        ch.set_time_mode(1)
        ch.run(800, 256)
        assert s.state(0)[3]["time"] == ch.counters()["time"]
    finally:
        s.close()


@pytest.mark.parametrize("L,R,cluster", [(40, 8, 2), (48, 8, 4)])
def test_cubic_binary32_beyond_one_cta(B, L, R, cluster):
    reps = [_cubic(L=L, r_max=3, T=0.05, seed=s, replica=s) for s in range(R)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=512)
    try:
        sh = B.cg_group_shape(s.h, 0)
        assert sh["cluster"] == cluster
        s.run(3 * 512 + 40, 1024)
        for k in (0, R - 1):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - ref.site_energies_fft3(n, phi, 0.5, L)).max() <= 1e-4
            o = s.observables(k)
            assert o["refreshes"] == 3 and o["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()


@pytest.mark.parametrize("R,kind", [(2, 0), (8, 2), (3, 1)], ids=["fft", "bf16x2", "fp64"])
def test_cubic_l64_binary32_without_the_table(B, R, kind):
    # L = 64 (N = 262144): the (L/2+1)^3 folded table (144 KiB) fits beside
    # no share of eps, and the cluster kernel's update reads 1/r indexed by
    # r^2 (12 KiB), so the replicas run on 8-CTA clusters (128 KiB of eps
    # each).  The set-up eps (binary64 sums, the table read from global
    # memory) equals the definition; every logged hop moves an electron from
    # an occupied site to an empty one within r_max; eps stays within 1e-4
    # of its definition, refreshed by the FFT, on the tensor cores or in
    # binary64 (refresh_kind 0, 2, 1).  (The r^2 table is the cubic cluster
    # kernel's for every L: the binary64 cluster trajectories above check it
    # hop for hop.)
    L, r_max = 64, 3
    reps = [_cubic(L=L, r_max=r_max, T=0.05, seed=s, replica=s) for s in range(R)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=2048, torch_memory=False,
                 refresh_kind=kind)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] == 8
        n0, eps0, phi0, _ = s.state(R - 1)
        assert np.abs(eps0 - ref.site_energies_fft3(n0, phi0, 0.5, L)).max() <= 1e-5
        rc, log = s.run_logged(2 * 2048 + 100, 1024)
        assert rc == B.CG_OK
        for k in (0, R - 1):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - ref.site_energies_fft3(n, phi, 0.5, L)).max() <= 1e-4
            o = s.observables(k)
            assert o["refreshes"] == 2 and o["max_eps_err_last_refresh"] <= 1e-4
        # replay replica 0's hops on its initial occupation (a fresh handle
        # rebuilds the same initial state)
        t = B.System(reps[:1], precision=B.CG_FP32, torch_memory=False)
        try:
            occ = t.state(0)[0].astype(np.int8).copy()
        finally:
            t.close()
        for e in log[0]:
            i, j = int(e["i"]), int(e["j"])
            assert occ[i] == 1 and occ[j] == 0
            d = [((j // L**a) % L - (i // L**a) % L + L // 2) % L - L // 2 for a in range(3)]
            assert 0 < d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= r_max * r_max
            occ[i], occ[j] = 0, 1
        np.testing.assert_array_equal(occ, s.state(0)[0])
    finally:
        s.close()


@pytest.mark.parametrize("kw", [dict(precision=0), dict(precision=1, pair_frac=0.2,
                                                                pair_rmax=2)])
def test_cubic_l64_refuses_what_does_not_fit(B, kw):
    # binary64 eps of the 64^3 lattice (2 MiB) outgrows 8 CTAs, and the
    # table-free kernel takes single hops only
    with pytest.raises(B.CgError, match="does not fit"):
        B.System([_cubic(L=64, r_max=3)], torch_memory=False, **kw)
