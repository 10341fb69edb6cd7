"""GPU checks of the batched state I/O (cg_group_replicas, cg_read_group_state,
cg_write_group_state): one copy per array for every replica of one lattice
size.  The paper has no counterpart; these calls checkpoint and resume a
batch.  A group read equals the per-replica reads; a batch resumed in a new
handle from a group checkpoint continues the same binary64 chains bit for
bit (and equals the serial oracle); an occupation with the wrong electron
count is refused and nothing is written; binary32 eps moves as float32.
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


def _mixed(R=10, T=0.05):
    sizes = [32, 16, 48]
    return [dict(L=sizes[k % 3], nu=0.5, W=1.0, xi=1.0, r_max=6 if sizes[k % 3] > 16 else 4,
                 T=T, E=0.01, seed=70 + k, replica=k) for k in range(R)]


def _unpack(words, N):
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    return bits[:N]


def test_group_read_equals_per_replica_reads(B):
    reps = _mixed()
    s = B.System(reps, precision=B.CG_FP64)
    try:
        s.run(300, 1024)
        seen = []
        for g in range(B.cg_num_groups(s.h)):
            idx = B.cg_group_replicas(s.h, g)
            L = B.cg_group_shape(s.h, g)["L"]
            assert all(reps[k]["L"] == L for k in idx) and list(idx) == sorted(idx)
            seen += list(idx)
            occ, eps, cnt = s.read_group(g)
            for m, k in enumerate(idx):
                n, e, _, c = s.state(int(k))
                np.testing.assert_array_equal(_unpack(occ[m], L * L), n)
                np.testing.assert_array_equal(_bits(eps[m]), _bits(e))
                assert {f: cnt[m][f] for f in cnt.dtype.names} == c
        assert sorted(seen) == list(range(len(reps)))
    finally:
        s.close()


def test_resume_from_group_checkpoint_is_bit_exact(B):
    reps = _mixed()
    a = B.System(reps, precision=B.CG_FP64)
    b = B.System(reps, precision=B.CG_FP64)
    try:
        a.run(250, 1024)
        for g in range(B.cg_num_groups(a.h)):
            occ, eps, cnt = a.read_group(g)
            # b has its own phi: the same seeds give the same disorder
            b.write_group(g, occ=occ, eps=eps, counters=cnt)
        a.run(300, 1024)
        b.run(300, 1024)
        for k in range(len(reps)):
            sa, sb = a.state(k), b.state(k)
            np.testing.assert_array_equal(sa[0], sb[0])
            np.testing.assert_array_equal(_bits(sa[1]), _bits(sb[1]))
            for f in ("rounds", "hops", "attempts", "P"):
                assert sa[3][f] == sb[3][f]
        # and both equal the serial chain
        p = reps[1]
        ch = oracle.Chain(p["L"], nu=0.5, W=1.0, xi=1.0, r_max=p["r_max"], T=p["T"], E=p["E"],
                          seed=p["seed"], replica=p["replica"])
        ch.run(550, 1024)
        np.testing.assert_array_equal(_bits(b.state(1)[1]), _bits(ch.state()[1]))
    finally:
        a.close()
        b.close()


def test_wrong_electron_count_is_refused_and_nothing_written(B):
    reps = _mixed(6)
    s = B.System(reps, precision=B.CG_FP64)
    try:
        g = 0
        occ, eps, cnt = s.read_group(g)
        bad = occ.copy()
        bad[-1, 0] ^= 1                      # one electron added or removed
        with pytest.raises(B.CgError) as ei:
            s.write_group(g, occ=bad, eps=eps)
        assert ei.value.code == B.CG_ESTATE
        occ2, eps2, _ = s.read_group(g)
        np.testing.assert_array_equal(occ2, occ)
        np.testing.assert_array_equal(_bits(eps2), _bits(eps))
    finally:
        s.close()


def test_binary32_group_io_moves_float32(B):
    reps = [dict(L=64, nu=0.5, W=2.0, xi=1.0, r_max=6, T=0.02, E=0.005, seed=s, replica=s)
            for s in range(12)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=512)
    try:
        s.run(700, 2048)
        occ, eps, cnt = s.read_group(0)
        assert eps.dtype == np.float32 and eps.shape == (12, 64 * 64)
        for k in (0, 11):
            e64 = s.state(k)[1]
            np.testing.assert_array_equal(eps[k].astype(np.float64), e64)
        eps2 = eps.copy()
        eps2[3] += np.float32(0.25)
        s.write_group(0, eps=eps2)
        np.testing.assert_array_equal(s.read_group(0)[1], eps2)
    finally:
        s.close()
