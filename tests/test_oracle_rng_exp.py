"""Pins of the oracle's Philox-4x32-10 and exp against outside references.

* Philox: cuRAND's host-side PHILOX4_32_10 generator (libcurand, CPU only).
  Its raw output block b comes from counter (lo32(b >> 16), hi32(b >> 16),
  b & 0xFFFF, 0) under key (seed lo 32, seed hi 32); reaching offsets past
  2^48 blocks exercises counter words 0, 1, 2 and both key words.
* exp: Python's ``math.exp`` (the platform libm) within 2 ulp.
* Uniformity and independence of the outputs by chi-square tests.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle

_CURAND_PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10


def _curand():
    for name in ("libcurand.so", "libcurand.so.10",
                 "/usr/local/cuda/lib64/libcurand.so",
                 "/usr/local/cuda/lib64/libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_words(cr, seed, n_words, offset_words=0):
    g = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(g), _CURAND_PHILOX) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        if offset_words:
            assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, np.uint32)
        rc = cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                               ctypes.c_size_t(n_words))
        assert rc == 0
        return out
    finally:
        cr.curandDestroyGenerator(g)


SEEDS = [0, 1, 0xFFFFFFFF, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0xDEADBEEF00000000]


@pytest.mark.parametrize("seed", SEEDS)
def test_philox_matches_curand_host_generator(seed):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = _curand_words(cr, seed, 4 * 128).reshape(-1, 4)
    for b in range(128):
        np.testing.assert_array_equal(oracle.philox([0, 0, b, 0], key), out[b])
    # offsets that move counter words 0 and 1
    for blocks in (65536 * 5 + 7, (1 << 48), (1 << 48) * 3 + 65536 * 9 + 11,
                   (1 << 61) + 65536 * 0xABCD + 0x1234):
        o = _curand_words(cr, seed, 4, offset_words=4 * blocks)
        hi, sub = blocks >> 16, blocks & 0xFFFF
        ctr = [hi & 0xFFFFFFFF, hi >> 32, sub, 0]
        np.testing.assert_array_equal(oracle.philox(ctr, key), o)


def test_philox_counter_word3_changes_output():
    # word 3 is not reachable through cuRAND's host generator (its device
    # generator reaches it: tests/test_gpu_philox_curand.py); here only that
    # it is consumed (distinct replicas give distinct streams)
    key = [7, 9]
    a = oracle.philox([1, 2, 3, 0], key)
    b = oracle.philox([1, 2, 3, 1], key)
    assert not np.array_equal(a, b)


def test_philox_uniformity_chi2():
    # 4096 blocks of counter (k, r, 0, 0): bytes of each word are uniform
    key = [0x12345678, 0x9ABCDEF0]
    words = np.array([oracle.philox([k, 5, 0, 0], key) for k in range(4096)],
                     dtype=np.uint32)
    for w in range(4):
        top = (words[:, w] >> 28).astype(np.int64)   # 16 bins
        cnt = np.bincount(top, minlength=16)
        exp = len(top) / 16
        chi2 = float(((cnt - exp) ** 2 / exp).sum())
        assert chi2 < 45.0  # 15 dof, p ~ 1e-4


def test_philox_independence_chi2():
    # joint 8 x 8 histograms of the top three bits of two outputs, against
    # independence: two words of one block, word 0 of consecutive labels k,
    # k + 1 (counter word 0) and of consecutive rounds r, r + 1 (counter word
    # 1), and words 2 and 3 of one block under the replica word set (counter
    # word 3).  A counter word the generator ignored or a word it repeated
    # would put every pair on the diagonal.
    key = [0x0BADF00D, 0x5EED1234]
    n = 8192

    def chi2(a, b):
        cnt = np.bincount((a >> 29).astype(np.int64) * 8 + (b >> 29).astype(np.int64),
                          minlength=64)
        exp = len(a) / 64
        return float(((cnt - exp) ** 2 / exp).sum())

    blk = np.array([oracle.philox([k, 9, 0, 0], key) for k in range(n + 1)], dtype=np.uint32)
    nxt = np.array([oracle.philox([77, r + 1, 0, 0], key) for r in range(n)], dtype=np.uint32)
    cur = np.array([oracle.philox([77, r, 0, 0], key) for r in range(n)], dtype=np.uint32)
    rep = np.array([oracle.philox([k, 9, 0, 3], key) for k in range(n)], dtype=np.uint32)
    # 63 degrees of freedom: the 1e-4 upper quantile is 113.5
    assert chi2(blk[:n, 0], blk[:n, 1]) < 113.5
    assert chi2(blk[:n, 0], blk[1:, 0]) < 113.5
    assert chi2(cur[:, 0], nxt[:, 0]) < 113.5
    assert chi2(rep[:, 2], rep[:, 3]) < 113.5
    # the statistic does see dependence: a word against itself
    assert chi2(blk[:n, 0], blk[:n, 0]) > 1000.0


def _ulp(x):
    return math.ulp(x)


def test_cg_exp_within_two_ulp_of_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([-23.0 * rng.random(20000), -np.logspace(-12, 1.3, 2000),
                         [0.0, -0.5, -1.0, -math.log(2), -23.0]])
    worst = 0.0
    for x in xs:
        got = oracle.cg_exp(float(x))
        ref = math.exp(float(x))
        worst = max(worst, abs(got - ref) / _ulp(ref))
    assert worst <= 2.0, worst


def test_exp_core_full_range():
    rng = np.random.default_rng(2)
    xs = -700.0 * rng.random(5000)
    for x in xs:
        got = oracle.exp_core(float(x))
        ref = math.exp(float(x))
        assert abs(got - ref) <= 2.0 * _ulp(ref), (x, got, ref)


def test_cg_exp_cutoff_keeps_every_decision():
    # exp(x) for x < -23 is returned as 0; the smallest acceptance variate is
    # (0 + 1/2) 2^-32 = 2^-33 > e^-23, so u < exp(x) is false either way.
    assert oracle.cg_exp(-23.0000001) == 0.0
    assert math.exp(-23.0) < 2.0 ** -33
    assert oracle.cg_exp(0.0) == 1.0
    # exp(-k ln2) = 2^-k up to the rounding of the argument k * ln2
    for k in range(1, 30):
        assert abs(oracle.cg_exp(-k * math.log(2)) / 2.0 ** -k - 1.0) <= 2e-16 * (k + 1)
