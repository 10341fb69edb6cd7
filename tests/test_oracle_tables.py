"""Pins of the oracle's geometry, 1/r table and tower weights.

Closed forms: lattice-point counts of the disk (Gauss circle problem), exact
values of the minimum-image 1/r, the shell symmetry of the tunnelling weights
exp(-2r/xi), and the normalisation of the integer tower.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("r_max,V", [(1, 4), (2, 12), (3, 28), (4, 48), (6, 112),
                                     (8, 196), (10, 316)])
def test_vector_count_is_gauss_circle(r_max, V):
    # number of nonzero integer points with x^2 + y^2 <= r^2: N(r) - 1 with
    # N(1..10) = 5, 13, 29, 49, 81, 113, 149, 197, 253, 317
    c = oracle.Chain(max(32, 2 * r_max + 2), r_max=r_max)
    assert c.V == V


def test_tinv_exact_values():
    c = oracle.Chain(16, r_max=4)
    assert c.tinv(0, 0) == 0.0
    assert c.tinv(1, 0) == 1.0
    assert c.tinv(0, 1) == 1.0
    assert c.tinv(2, 0) == 0.5
    assert c.tinv(3, 4) == 0.2
    # 1/r is one rounded sqrt and one rounded divide: within 1 ulp of the
    # exact value (exact for the perfect squares above)
    getcontext().prec = 60
    for fx, fy in [(1, 1), (1, 2), (2, 3), (5, 7), (8, 8)]:
        exact = Decimal(1) / Decimal(fx * fx + fy * fy).sqrt()
        got = c.tinv(fx, fy)
        assert abs(Decimal(got) - exact) <= Decimal(math.ulp(got))
    # minimum image: L-1 is distance 1, L/2 is the farthest
    assert c.tinv(15, 0) == 1.0
    assert c.tinv(-15, 0) == 1.0
    assert c.tinv(8, 8) == 1.0 / math.sqrt(128.0)
    assert c.tinv(-3, 5) == c.tinv(5, 3) == c.tinv(3, -5)


def test_tinv_matches_hypot_everywhere():
    L = 12
    c = oracle.Chain(L, r_max=2)
    t = c.tinv_table()
    for fy in range(L // 2 + 1):
        for fx in range(L // 2 + 1):
            if fx == fy == 0:
                assert t[fy, fx] == 0.0
            else:
                assert abs(t[fy, fx] - 1.0 / math.hypot(fx, fy)) <= 1e-16


@pytest.mark.parametrize("r_max,xi", [(4, 1.0), (6, 1.0), (8, 1.0), (10, 1.5), (3, 0.7)])
def test_tower_weights(r_max, xi):
    c = oracle.Chain(32, r_max=r_max, xi=xi)
    dx, dy, Wi, w = c.vectors()
    r = np.hypot(dx, dy)
    # real weights are exp(-2 r / xi)
    np.testing.assert_allclose(w, np.exp(-2.0 * r / xi), rtol=4e-16, atol=0)
    assert abs(c.Z - math.fsum(w)) <= 1e-15 * c.Z
    # equal weights within a shell, so Q is symmetric under d -> -d
    for k in range(len(dx)):
        same = (dx * dx + dy * dy) == dx[k] ** 2 + dy[k] ** 2
        assert len(set(Wi[same].tolist())) == 1
        kk = np.where((dx == -dx[k]) & (dy == -dy[k]))[0]
        assert len(kk) == 1 and Wi[kk[0]] == Wi[k]
    S = int(Wi.sum(dtype=np.uint64))
    assert S <= 2 ** 32
    assert 2 ** 32 - S <= len(dx)
    # integer weights are the floor of 2^32 w / Z
    for k in range(len(dx)):
        exact = Fraction(w[k]) / Fraction(c.Z) * 2 ** 32
        assert abs(int(Wi[k]) - exact) <= 1 + 1e-6
    # ordering: dy outer ascending, dx inner ascending
    order = list(zip(dy.tolist(), dx.tolist()))
    assert order == sorted(order)
    assert c.Gamma == c.N * c.Z


def test_disk_fits_inside_half_lattice():
    with pytest.raises(ValueError):
        oracle.Chain(8, r_max=4)    # r_max must be < L/2
    oracle.Chain(10, r_max=4)
