"""GPU checks of the binary32 form (eps in binary32, periodic binary64 refresh).

The binary32 form is not bit-exact by design; it is checked against what the
definition of eps fixes and against the serial chain's law:

* the initial binary32 eps is the oracle's binary64 eps rounded to binary32;
* after a run, eps stays within 1e-4 of phi + G (n - nu) evaluated by numpy on
  the chain's own configuration (any configuration must satisfy it), and the
  refresh's reported maximum error agrees;
* over 64 disorder samples, the energy per site, dipole drift and acceptance
  of the binary32 form agree with the serial binary64 oracle within three
  standard errors of the paired differences (same disorder and start,
  disjoint random numbers, so the pairs are independent trajectories).
"""
import math

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


def _oracle_for(p):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0))


@pytest.mark.parametrize("L", [16, 48, 128])
def test_initial_eps_is_rounded_binary64(B, L):
    p = dict(L=L, nu=0.5, W=2.0, xi=1.0, r_max=6, T=0.01, E=0.005, seed=3)
    s = B.System([p], precision=B.CG_FP32)
    try:
        n, eps, phi, _ = s.state(0)
        on, oeps, ophi = _oracle_for(p).state()
        np.testing.assert_array_equal(n, on)
        np.testing.assert_array_equal(eps, oeps.astype(np.float32).astype(np.float64))
    finally:
        s.close()


@pytest.mark.parametrize("L,T,hops,every", [(32, 0.02, 20000, 1024), (64, 0.01, 12000, 1024),
                                            (128, 0.01, 6000, 1024)])
def test_eps_error_stays_below_1em4(B, L, T, hops, every):
    reps = [dict(L=L, nu=0.5, W=2.0, xi=1.0, r_max=8 if L >= 64 else 6, T=T, E=0.005,
                 seed=s, replica=s) for s in range(3)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=every)
    try:
        s.run(hops + 300, 4096)         # ends 300 hops after a refresh
        for k in range(len(reps)):
            n, eps, phi, c = s.state(k)
            exact = ref.site_energies_fft(n, phi, 0.5, L)
            err = np.abs(eps - exact).max()
            assert err <= 1e-4, err
            obs = s.observables(k)
            assert obs["refreshes"] >= 1
            assert 0 < obs["max_eps_err_last_refresh"] <= 1e-4
            # running energy stays consistent with Eq. 1 on the final state
            H = float(phi @ n + 0.5 * (n - 0.5) @ (exact - phi)) - 0.005 * c["P"]
            assert abs(c["energy"] - H) <= 1e-3 * (1 + abs(H) / L ** 2)
    finally:
        s.close()


def test_refresh_restores_exact_eps(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=4)
    s = B.System([p], precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_FP64)
    try:
        s.run(5000, 1024)
        B.cg_refresh(s.h)
        n, eps, phi, _ = s.state(0)
        exact = ref.site_energies_fft(n, phi, 0.5, 32)
        # after a refresh eps is the binary64 value rounded to binary32
        assert np.abs(eps - exact).max() <= 4e-7 * max(1.0, np.abs(exact).max())
    finally:
        s.close()


def test_observables_agree_with_binary64_oracle_over_64_samples(B):
    # same disorder and random start on both sides, independent trajectories:
    # the GPU replicas' round counter starts at 2^40, so their labels draw
    # Philox counters the oracle's chains (round 0 onwards) never reach
    L, T, E, hops, M = 32, 0.05, 0.02, 3000, 1024
    seeds = list(range(64))
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=T, E=E, seed=s, replica=s)
            for s in seeds]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=1024)
    try:
        for k in range(len(seeds)):
            n, eps, phi, c = s.state(k)
            c["rounds"] = 1 << 40
            B.cg_write_state(s.h, k, n, eps=eps, phi=phi, counters=c)
        s.run(hops, M)
        g = np.array([[o["energy_per_site"], o["P"], o["acceptance"]]
                      for o in (s.observables(k) for k in range(len(seeds)))])
    finally:
        s.close()
    o = []
    for p in reps:
        ch = _oracle_for(p)
        ch.run(hops, M)
        c = ch.counters()
        o.append([c["energy"] / L ** 2, c["P"], c["hops"] / c["attempts"]])
    o = np.array(o)
    d = g - o
    for col, name in enumerate(["E/N", "P", "A"]):
        se = d[:, col].std(ddof=1) / math.sqrt(len(seeds))
        mean = d[:, col].mean()
        assert se > 0, name
        assert abs(mean) <= 3 * se, (name, mean, se)


@pytest.mark.parametrize("L,R", [(32, 20), (48, 9), (64, 40), (128, 300), (16, 513)])
def test_tensor_core_refresh_matches_definition(B, L, R):
    # split-BF16 G (2n - 1) on the tensor cores: eps = phi + D/2 + (1/2 - nu) C0;
    # R = 300 exercises two N sub-tiles (256 + 48), R = 513 two launches
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.05, E=0.01, seed=s, replica=s)
            for s in range(R)]
    s = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_BF16X2)
    try:
        s.run(50, 256)
        B.cg_refresh(s.h)
        worst = 0.0
        for k in sorted({0, 1, R // 2, R - 1}):
            n, eps, phi, _ = s.state(k)
            exact = ref.site_energies_fft(n, phi, 0.5, L)
            worst = max(worst, float(np.abs(eps - exact).max()))
            obs = s.observables(k)
            assert obs["refreshes"] == 1
            assert obs["max_eps_err_last_refresh"] <= 1e-4
        assert worst <= 5e-5, worst
    finally:
        s.close()


def test_tensor_core_refresh_in_runs(B):
    # 64 replicas refreshed every 512 hops on the tensor cores stay within 1e-4
    reps = [dict(L=64, nu=0.5, W=2.0, xi=1.0, r_max=6, T=0.01, E=0.005, seed=s, replica=s)
            for s in range(64)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=512,
                 refresh_kind=B.CG_REFRESH_BF16X2)
    try:
        s.run(4 * 512 + 100, 4096)
        for k in (0, 31, 63):
            n, eps, phi, _ = s.state(k)
            exact = ref.site_energies_fft(n, phi, 0.5, 64)
            assert np.abs(eps - exact).max() <= 1e-4
            assert s.observables(k)["refreshes"] == 4
    finally:
        s.close()
