"""GPU checks of the FFT refresh of binary32 eps (the convolution theorem:
eps - phi = IDFT(DFT(n - nu) DFT(g)), g the minimum-image 1/r, two replicas
per complex binary32 transform).

After hops from the random start, a refresh rebuilds eps within 2e-5 of the
definition (evaluated in binary64 by numpy's FFT) on square and cubic
lattices of sides 2^m and 3 2^m, with an even and an
odd number of replicas (the last one alone in its transform), reports the
largest change and counts the refresh; it agrees with the binary64 direct
refresh on the same states; inside runs it keeps eps within 1e-4; the
automatic choice takes it for those sides, and the other kinds stay
reachable.
"""
import numpy as np
import pytest

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


def _reps(L, R, dim=2, r_max=3, T=0.05):
    return [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=r_max, T=T, E=0.01, seed=s, replica=s,
                 dim=dim) for s in range(R)]


def _exact(n, phi, L, dim):
    return (ref.site_energies_fft3(n, phi, 0.5, L) if dim == 3
            else ref.site_energies_fft(n, phi, 0.5, L))


@pytest.mark.parametrize("L,dim,R", [(4, 2, 1), (8, 2, 2), (16, 2, 3), (64, 2, 5),
                                     (128, 2, 20), (256, 2, 3), (8, 3, 3), (16, 3, 2),
                                     (32, 3, 7), (64, 3, 2),
                                     # L = 3 2^m: the radix-3 step, then 2^m-point
                                     (6, 2, 1), (12, 2, 3), (48, 2, 4), (96, 2, 5),
                                     (192, 2, 2), (6, 3, 3), (12, 3, 2), (24, 3, 3),
                                     (48, 3, 2)])
def test_fft_refresh_matches_definition(B, L, dim, R):
    r_max = 1 if L == 4 else 2 if L == 6 else 3
    reps = _reps(L, R, dim, r_max)
    s = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_FFT, torch_memory=False)
    try:
        assert s.run(200, 512) == B.CG_OK
        B.cg_refresh(s.h)
        worst = 0.0
        for k in sorted({0, R // 2, R - 1}):
            n, eps, phi, _ = s.state(k)
            worst = max(worst, float(np.abs(eps - _exact(n, phi, L, dim)).max()))
            o = s.observables(k)
            assert o["refreshes"] == 1
            assert 0 < o["max_eps_err_last_refresh"] <= 1e-4
        assert worst <= 2e-5, worst
    finally:
        s.close()


@pytest.mark.parametrize("L,dim", [(32, 2), (16, 3)])
def test_fft_refresh_agrees_with_binary64_refresh(B, L, dim):
    # the same chains (same seeds, same hops) refreshed both ways
    reps = _reps(L, 4, dim)
    a = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_FFT)
    b = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_FP64)
    try:
        for s in (a, b):
            assert s.run(300, 1024) == B.CG_OK
            B.cg_refresh(s.h)
        for k in range(4):
            na, ea, _, _ = a.state(k)
            nb, eb, _, _ = b.state(k)
            np.testing.assert_array_equal(na, nb)
            assert np.abs(ea - eb).max() <= 2e-5
    finally:
        a.close()
        b.close()


def test_fft_refresh_in_runs_is_the_automatic_choice(B):
    # 6 replicas of L = 64 refreshed every 256 hops: the automatic choice
    # (power-of-two L) is the FFT, so even a group below the tensor-core
    # batch size refreshes by it
    reps = _reps(64, 6, 2, 6, 0.03)
    s = B.System(reps, precision=B.CG_FP32, refresh_every=256)
    try:
        assert s.run(4 * 256 + 50, 1024) == B.CG_OK
        for k in (0, 5):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - _exact(n, phi, 64, 2)).max() <= 1e-4
            o = s.observables(k)
            assert o["refreshes"] == 4 and 0 < o["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()


def test_fft_refresh_at_the_bench_batch_size(B):
    # the bench's batch: 304 replicas of L = 128 (152 complex transforms per
    # pass); after 1024 hops and a refresh, sampled replicas' eps is within
    # 2e-5 of the definition and every replica counted one refresh
    reps = [dict(L=128, nu=0.5, W=2.0, xi=1.0, r_max=8, T=0.01, E=0.005, seed=s, replica=s)
            for s in range(304)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=1024, block_threads=512)
    try:
        assert s.run(1024, 4096) == B.CG_OK
        for k in (0, 151, 152, 303):
            n, eps, phi, _ = s.state(k)
            assert np.abs(eps - _exact(n, phi, 128, 2)).max() <= 2e-5
            o = s.observables(k)
            assert o["refreshes"] == 1 and 0 < o["max_eps_err_last_refresh"] <= 1e-4
    finally:
        s.close()


@pytest.mark.parametrize("L,dim,n_occ", [(12, 2, 48), (48, 2, 768), (24, 3, 4608)])
def test_fft_refresh_with_a_filling_binary32_does_not_hold(B, L, dim, n_occ):
    # nu = 1/3 is not a binary32 number; the transforms take n - nu_f and the
    # last pass adds (nu_f - nu) C0 back in binary64
    N = L ** dim
    nu = n_occ / N
    reps = [dict(r, nu=nu) for r in _reps(L, 3, dim, 2)]
    s = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_FFT)
    try:
        assert s.run(200, 512) == B.CG_OK
        B.cg_refresh(s.h)
        for k in range(3):
            n, eps, phi, _ = s.state(k)
            exact = (ref.site_energies_fft3(n, phi, nu, L) if dim == 3
                     else ref.site_energies_fft(n, phi, nu, L))
            assert np.abs(eps - exact).max() <= 2e-5
    finally:
        s.close()
