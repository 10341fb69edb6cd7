"""GPU checks of the thread-block-cluster form (eps split by rows over 2-8 CTAs).

* In binary64 the cluster kernel must reproduce the serial chain bit for bit,
  like the single-CTA kernel: forced clusters on small lattices are compared
  hop by hop with the oracle (all exchange paths: remote eps reads, candidate
  slots, the uniform stop decisions).
* L = 256 in binary32 (eps 256 KiB, beyond one CTA) picks a cluster by itself
  and keeps eps within 1e-4 of phi + G (n - nu).
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
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0))


# (16, 8): one base row per CTA (L = 2C), where the row-owner division has
# no 32-bit multiplier and takes the row index itself
@pytest.mark.parametrize("L,cluster,T", [(32, 2, 0.05), (64, 4, 0.02), (48, 2, 0.1),
                                         (64, 8, 0.05), (16, 8, 0.1)])
def test_cluster_binary64_trajectory_is_bit_exact(B, L, cluster, T):
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=T, E=0.01, seed=s, replica=s)
            for s in range(3)]
    s = B.System(reps, precision=B.CG_FP64, cluster_size=cluster)
    try:
        rc, log = s.run_logged(1500, 2048)
        assert rc == B.CG_OK
        for k, p in enumerate(reps):
            ch = _oracle_for(p)
            _, olog = ch.run(1500, 2048, log=True)
            for f in ("i", "j", "q", "p", "round", "dx", "dy"):
                np.testing.assert_array_equal(log[k][f], olog[f], err_msg=f)
            np.testing.assert_array_equal(_bits(log[k]["dE"]), _bits(olog["dE"]))
            n, eps, phi, c = s.state(k)
            on, oeps, _ = ch.state()
            np.testing.assert_array_equal(n, on)
            np.testing.assert_array_equal(_bits(eps), _bits(oeps))
            oc = ch.counters()
            for f in ("rounds", "hops", "attempts", "P"):
                assert c[f] == oc[f], f
    finally:
        s.close()


def test_cluster_constant_acceptance_matches_oracle(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=3)
    s = B.System([p], precision=B.CG_FP64, cluster_size=4)
    try:
        B.cg_set_toy_acceptance(s.h, 3e-4)
        _, log = s.run_logged(300, 4096)
        ch = _oracle_for(p)
        ch.set_toy(3e-4)
        _, olog = ch.run(300, 4096, log=True)
        for f in ("q", "p", "round", "i"):
            np.testing.assert_array_equal(log[0][f], olog[f])
    finally:
        s.close()


@pytest.mark.parametrize("cluster", [2, 4])
def test_cluster_hop_time_limit_returns_timeout(B, cluster):
    # a hop that never ends (no label accepts, unbounded rounds): rank 0's
    # wall clock passes the limit, every CTA of the cluster reads that
    # decision from rank 0's exchange slot after the same cluster barrier and
    # the launch stores a valid state
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=3)
    s = B.System([p], precision=B.CG_FP64, cluster_size=cluster, hop_timeout_ms=200)
    try:
        assert B.cg_group_shape(s.h, 0)["cluster"] == cluster
        n0, e0, _, c0 = s.state(0)
        B.cg_set_toy_acceptance(s.h, 0.0)
        with pytest.raises(B.CgError) as ei:
            s.run(1, 1024)
        assert ei.value.code == B.CG_ETIMEOUT
        n1, e1, _, c1 = s.state(0)
        np.testing.assert_array_equal(n0, n1)
        np.testing.assert_array_equal(_bits(e0), _bits(e1))
        assert c1["hops"] == c0["hops"]
        # complete failed rounds only: M attempts and one round each
        assert c1["rounds"] > c0["rounds"]
        assert c1["attempts"] - c0["attempts"] == 1024 * (c1["rounds"] - c0["rounds"])
        # the handle keeps working and still follows the serial chain
        B.cg_set_toy_acceptance(s.h, -1.0)
        _, log = s.run_logged(50, 256)
        ch = _oracle_for(p)
        ch.set_counters(dict(c1))
        _, olog = ch.run(50, 256, log=True)
        for f in ("i", "j", "q", "p", "round"):
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
    finally:
        s.close()


def test_l256_binary32_cluster_keeps_eps_within_1em4(B):
    reps = [dict(L=256, nu=0.5, W=1.0, xi=1.5, r_max=10, T=0.02, E=0.005, seed=s, replica=s)
            for s in range(2)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=512,
                 refresh_kind=B.CG_REFRESH_BF16X2)
    try:
        s.run(2 * 512 + 200, 4096)
        for k in range(2):
            n, eps, phi, c = s.state(k)
            assert int(n.sum()) == 256 * 256 // 2
            exact = ref.site_energies_fft(n, phi, 0.5, 256)
            assert np.abs(eps - exact).max() <= 1e-4
            obs = s.observables(k)
            assert obs["refreshes"] == 2 and obs["hops"] == 2 * 512 + 200
            assert obs["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()
