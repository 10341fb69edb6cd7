"""The binary32 form (binary32 eps with a periodic refresh, binary64 near
ties) against the binary64 form on the extensions: the cubic lattice (with
the binary16-split tensor-core refresh) and two-electron hops.  The same
disorder samples run from their common random start in both forms; the
paired differences of E/N, P and the acceptance over the samples are
consistent with zero (|z| below 3.5 each), and eps stays within 1e-4 of its
definition at every refresh.  The binary32 chains draw from a disjoint
part of each replica's random stream, so the two forms' trajectories are
independent and the paired differences carry statistical noise, not only
the forms' rounding.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROUND_SHIFT = 1 << 40


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def _paired_z(B, reps, hops, M, **kw):
    # both forms start from the samples' common random configuration; the
    # binary32 chains draw from a disjoint part of each replica's random
    # stream (round counter + 2^40), so the pairs share their disorder but
    # not their trajectories, and each z is a paired two-sample statistic
    vals = {}
    max_err = 0.0
    for key, prec in (("fp32", B.CG_FP32), ("fp64", B.CG_FP64)):
        s = B.System(reps, precision=prec, refresh_every=512 if prec == B.CG_FP32 else 0, **kw)
        try:
            if prec == B.CG_FP32:
                for k in range(len(reps)):
                    n, _, phi, c = s.state(k)
                    c = dict(c)
                    c["rounds"] += ROUND_SHIFT
                    B.cg_write_state(s.h, k, n, phi=phi, counters=c)
            assert s.run(hops, M) == B.CG_OK
            obs = [s.observables(k) for k in range(len(reps))]
        finally:
            s.close()
        vals[key] = np.array([[o["energy_per_site"], o["P"], o["acceptance"]] for o in obs])
        if prec == B.CG_FP32:
            max_err = max(o["max_eps_err_last_refresh"] for o in obs)
    d = vals["fp32"] - vals["fp64"]
    n = len(reps)
    z = []
    for col in range(3):
        se = d[:, col].std(ddof=1) / math.sqrt(n)
        assert se > 0, col                  # independent trajectories, not copies
        z.append(d[:, col].mean() / se)
    return np.array(z), max_err


def test_cubic_binary32_observables_match_binary64(B):
    reps = [dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.05, E=0.01, seed=s, replica=s,
                 dim=3) for s in range(48)]
    z, max_err = _paired_z(B, reps, 6000, 1024, refresh_kind=B.CG_REFRESH_BF16X2)
    assert np.all(np.abs(z) < 3.5), z
    assert max_err <= 1e-4


def test_pair_hop_binary32_observables_match_binary64(B):
    reps = [dict(L=32, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.1, E=0.01, seed=s, replica=s)
            for s in range(48)]
    z, max_err = _paired_z(B, reps, 6000, 1024, pair_frac=0.2, pair_rmax=4)
    assert np.all(np.abs(z) < 3.5), z
    assert max_err <= 1e-4
