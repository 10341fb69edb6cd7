"""GPU checks of the density-of-states observable g(eps) (the single-particle
DOS whose Coulomb gap the paper discusses, section "Results for the lattice
model in two dimensions"): the device histogram equals, bin for bin, the
definition evaluated by numpy on the same energies (binary64 and binary32,
square and cubic lattices, a range narrower than the energies); in binary64
it equals the histogram of the serial oracle's energies after the same
chain; repeated calls add snapshots; a relaxed low-temperature state shows
the Coulomb gap at the chemical potential.
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


def _hist(eps, nbins, lo, hi):
    """The definition: x = (eps - lo) * (nbins / (hi - lo)) in binary64;
    counted in bin floor(x) when eps >= lo and x < nbins."""
    e = np.asarray(eps, dtype=np.float64)
    x = (e - lo) * (nbins / (hi - lo))
    keep = (e >= lo) & (x < nbins)
    return np.bincount(np.floor(x[keep]).astype(np.int64), minlength=nbins)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nbins,lo,hi", [(100, -1.5, 1.5), (4096, -0.3, 0.2), (7, 0.0, 0.5)])
def test_histogram_equals_the_definition(B, prec, nbins, lo, hi):
    reps = [dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=s, replica=s)
            for s in range(5)]
    reps.append(dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.05, E=0.0, seed=9, replica=9,
                     dim=3))
    precision = B.CG_FP64 if prec == "fp64" else B.CG_FP32
    s = B.System(reps, precision=precision, refresh_every=256 if prec == "fp32" else 0)
    try:
        s.run(700, 512)
        got = s.eps_histogram(nbins, lo, hi).cpu().numpy()
        want = sum(_hist(s.state(k)[1], nbins, lo, hi) for k in range(len(reps)))
        np.testing.assert_array_equal(got, want)
        # a subset of the replicas, and a second call adds to the same counts
        part = s.eps_histogram(nbins, lo, hi, first=2, count=3)
        part = s.eps_histogram(nbins, lo, hi, first=2, count=3, counts=part).cpu().numpy()
        want2 = sum(_hist(s.state(k)[1], nbins, lo, hi) for k in (2, 3, 4))
        np.testing.assert_array_equal(part, 2 * want2)
    finally:
        s.close()


def test_binary64_histogram_equals_the_oracle(B):
    p = dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=4, replica=0)
    s = B.System([p], precision=B.CG_FP64)
    try:
        s.run(2000, 1024)
        ch = oracle.Chain(32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01, seed=4)
        ch.run(2000, 1024)
        got = s.eps_histogram(64, -1.2, 1.2).cpu().numpy()
        np.testing.assert_array_equal(got, _hist(ch.state()[1], 64, -1.2, 1.2))
    finally:
        s.close()


def test_relaxed_state_shows_the_coulomb_gap(B):
    reps = [dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.02, E=0.0, seed=s, replica=s)
            for s in range(8)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=1024)
    try:
        nb, lo, hi = 40, -1.0, 1.0           # bins of width 0.05
        g0 = s.eps_histogram(nb, lo, hi).cpu().numpy()
        s.run(20000, 4096)
        g1 = s.eps_histogram(nb, lo, hi).cpu().numpy()
        centre = slice(19, 21)               # |eps| < 0.05
        shoulder = np.r_[26:28, 12:14]       # 0.3 <= |eps| < 0.4
        assert g0[centre].mean() > 0.5 * g0[shoulder].mean()      # no gap at the start
        assert g1[centre].mean() < 0.25 * g1[shoulder].mean()     # the Coulomb gap
    finally:
        s.close()


def test_histogram_rejects_bad_arguments(B):
    s = B.System([dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=0)])
    try:
        for bad in (dict(nbins=0, lo=0, hi=1), dict(nbins=5000, lo=0, hi=1),
                    dict(nbins=10, lo=1, hi=1), dict(nbins=10, lo=0, hi=1, first=1)):
            with pytest.raises(B.CgError):
                s.eps_histogram(**bad)
    finally:
        s.close()
