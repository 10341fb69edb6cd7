"""Pins of the oracle's stochastic time increment (reading R13 of the mixed
PR algorithm, step 3c: dt Gaussian with mean m/Gamma and standard deviation
sqrt(m)/Gamma, clamped at zero).

The project logarithm and cos(2 pi u) are checked against libm, the normal
deviates against the standard normal distribution (moments, tail mass, the
Kolmogorov-Smirnov distance, lag-1 correlation), the increment against its
closed forms, and a chain's stochastic time against the per-hop increments
recomputed from its hop log and against the deterministic clock
attempts / Gamma.
"""
import math

import numpy as np
import pytest

import oracle


def _ulp(x):
    return math.ulp(x)


def test_log_matches_libm_within_two_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([(rng.integers(0, 1 << 32, 20000) + 0.5) * 2.0 ** -32,
                         np.exp(-rng.random(5000) * 23.0),
                         1.0 - rng.random(2000) * 1e-6, [0.5, 0.75, 2.0 ** -33, 1.0 - 2.0 ** -33]])
    for x in xs:
        got, want = oracle.log(float(x)), math.log(float(x))
        assert abs(got - want) <= 2 * _ulp(want) + 1e-300, (x, got, want)
    assert oracle.log(1.0) == 0.0
    for k in range(-40, 41):
        # k ln 2 to within an ulp: the split constant makes k LN2_HI exact
        want = k * math.log(2.0)
        assert abs(oracle.log(2.0 ** k) - want) <= _ulp(want) + 1e-300, k


def test_cos2pi_matches_libm_and_exact_points():
    rng = np.random.default_rng(1)
    us = np.concatenate([rng.integers(0, 1 << 32, 20000) * 2.0 ** -32, [2.0 ** -32, 1 - 2.0 ** -32]])
    for u in us:
        got = oracle.cos2pi(float(u))
        want = math.cos(2.0 * math.pi * float(u))
        # libm's own argument 2 pi u carries a rounding of up to ulp(2 pi u)
        assert abs(got - want) <= 4e-16 + 2 * math.ulp(2 * math.pi * float(u)), (u, got, want)
    assert oracle.cos2pi(0.0) == 1.0
    assert oracle.cos2pi(0.25) == 0.0 and oracle.cos2pi(0.75) == 0.0
    assert oracle.cos2pi(0.5) == -1.0
    assert abs(oracle.cos2pi(0.125) - math.sqrt(0.5)) <= 2 * _ulp(math.sqrt(0.5))


def _normal_cdf(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def test_hop_deviates_are_standard_normal():
    n = 200_000
    z = np.array([oracle.gauss(11, 3, h) for h in range(n)])
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    tail = np.mean(np.abs(z) > 3.0)
    p3 = 2 * (1 - _normal_cdf(3.0))
    assert abs(tail - p3) < 5 * math.sqrt(p3 * (1 - p3) / n)
    zs = np.sort(z)
    F = np.array([_normal_cdf(v) for v in zs[:: 50]])
    emp = (np.arange(0, n, 50) + 1) / n
    assert np.max(np.abs(emp - F)) < 1.63 / math.sqrt(n) + 50 / n
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5 * se
    # a different replica or seed gives an independent sequence
    z2 = np.array([oracle.gauss(11, 4, h) for h in range(20000)])
    assert abs(np.corrcoef(z[:20000], z2)[0, 1]) < 5 / math.sqrt(20000)


def test_time_increment_closed_forms():
    G = 1234.5
    assert oracle.time_increment(G, 100, 0.0) == 100.0 / G
    assert oracle.time_increment(G, 100, 1.0) == (100.0 + 10.0) / G
    assert oracle.time_increment(G, 9, -2.0) == (9.0 - 6.0) / G
    assert oracle.time_increment(G, 1, -2.0) == 0.0          # clamped at zero
    assert oracle.time_increment(G, 4, -2.0) == 0.0


def _chain(mode):
    ch = oracle.Chain(24, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.02, seed=9)
    ch.set_time_mode(mode)
    return ch


def test_default_mode_keeps_the_deterministic_clock():
    ch = _chain(0)
    ch.run(500, 256)
    assert ch.counters()["time"] == 0.0


def test_stochastic_time_is_the_sum_of_the_hop_increments():
    ch = _chain(1)
    M, n = 256, 4000
    c0 = ch.counters()
    _, log = ch.run(n, M, log=True)
    c1 = ch.counters()
    G = ch.Gamma
    m = (log["p"].astype(np.int64) - 1) * M + log["q"].astype(np.int64)
    t = 0.0
    for h in range(n):
        t = t + oracle.time_increment(G, int(m[h]), oracle.gauss(9, 0, c0["hops"] + h))
    assert c1["time"] == t
    # the Gaussian has mean m / Gamma: the stochastic clock follows
    # attempts / Gamma within a few of its standard deviations sqrt(sum m)/Gamma
    att = c1["attempts"] - c0["attempts"]
    assert abs(c1["time"] - att / G) < 5 * math.sqrt(att) / G
    # the standardised increments (unclamped ones) have mean 0 and variance 1
    z = np.array([oracle.gauss(9, 0, c0["hops"] + h) for h in range(n)])
    keep = m + np.sqrt(m) * z > 0
    assert keep.mean() > 0.9
