"""The synthetic workloads name the five benchmark configurations of the
lattice model exactly: the bit-exact L=16 chain, the L=64 relaxation runs,
the L=128 low-temperature headline system, the batch of uneven L and the
L=256 cluster system.  The benchmark and the parity tests take their
parameters from these recipes, so a drift in any of them would change what
is measured without changing the code that measures it."""
from paper_1407_5026_gb300 import workloads as W


def _params(r):
    return (r.L, r.nu, r.W, r.xi, r.r_max, r.T, r.E, r.dim, r.sites)


def test_bit_exact_l16_chain():
    w = W.l16_fp64()
    (r,) = w.replicas
    # phi ~ U[-0.5, 0.5] is full width W = 1
    assert _params(r) == (16, 0.5, 1.0, 1.0, 4, 0.05, 0.0, 2, 0)
    assert (r.seed, r.replica) == (0, 0)
    assert (w.M, w.hops, w.precision, w.refresh_every) == (256, 10_000, "fp64", 0)


def test_l64_relaxation_runs():
    assert W.L64_TEMPERATURES == (0.02, 0.05, 0.1)
    assert W.L64_SEEDS == tuple(range(8))
    for T in W.L64_TEMPERATURES:
        for s in W.L64_SEEDS:
            w = W.l64_fp64(T=T, seed=s)
            (r,) = w.replicas
            assert _params(r) == (64, 0.5, 1.0, 1.0, 6, T, 0.01, 2, 0)
            assert r.seed == s
            assert (w.M, w.hops, w.precision) == (4096, 1_000_000, "fp64")


def test_l128_headline_system():
    # phi ~ U[-1, 1] is full width W = 2
    for prec, refresh in (("fp32", 1024), ("fp64", 0)):
        w = W.l128(precision=prec)
        (r,) = w.replicas
        assert _params(r) == (128, 0.5, 2.0, 1.0, 8, 0.01, 0.005, 2, 0)
        assert (w.hops, w.refresh_every) == (10_000_000, refresh)
    assert W.L128_M_SWEEP == (1024, 4096, 16384, 65536)
    b = W.l128_batch(304)
    assert len(b.replicas) == 304 and b.refresh_every == 1024
    assert {_params(r) for r in b.replicas} == {(128, 0.5, 2.0, 1.0, 8, 0.01, 0.005, 2, 0)}
    assert [r.seed for r in b.replicas] == list(range(304))
    assert len({(r.seed, r.replica) for r in b.replicas}) == 304


def test_batch_of_uneven_sizes():
    w = W.mixed_batch()
    assert len(w.replicas) == 256
    assert {r.L for r in w.replicas} == {32, 48, 64, 96}
    for r in w.replicas:
        assert _params(r)[1:] == (0.5, 1.0, 1.0, 6, 0.03, 0.01, 2, 0)
    # independent Philox streams: every replica its own seed
    assert len({r.seed for r in w.replicas}) == 256
    assert (w.precision, w.refresh_every) == ("fp32", 1024)
    # the draw of sizes is seeded: the same batch every time
    assert [r.L for r in W.mixed_batch().replicas] == [r.L for r in w.replicas]


def test_l256_cluster_system():
    w = W.l256()
    assert len(w.replicas) == 16
    assert {_params(r) for r in w.replicas} == {(256, 0.5, 1.0, 1.5, 10, 0.02, 0.005, 2, 0)}
    assert len({r.seed for r in w.replicas}) == 16
    assert (w.hops, w.precision, w.refresh_every) == (10_000_000, "fp32", 4096)
