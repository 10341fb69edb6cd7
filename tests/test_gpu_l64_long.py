"""The L=64 configuration in binary64 over a long run: all 24 chains of the
workload (T in {0.02, 0.05, 0.1} x seeds 0-7, field E=0.01, M=4096) run
1e5 hops each as one GPU batch, and each final state (occupation, eps bit
for bit) and its counters equal the serial oracle's after the same hops.
The oracle chains run in a process pool on the host cores (spawn start).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1407_5026_gb300 import workloads

pytestmark = pytest.mark.gpu

HOPS = 100_000


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def test_l64_long_runs_bit_exact(B):
    from tests import oracle_workers
    reps = []
    for T in workloads.L64_TEMPERATURES:
        for seed in range(8):
            reps.append(workloads.l64_fp64(T=T, seed=seed).replicas[0].as_dict())
    M = workloads.l64_fp64().M
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(reps), max(1, (os.cpu_count() or 2) - 1))) as pool:
        pending = pool.map_async(oracle_workers.run_chain, [(p, HOPS, M) for p in reps])
        s = B.System(reps, precision=B.CG_FP64)
        try:
            assert s.run(HOPS, M) == B.CG_OK
            got = [s.state(k) for k in range(len(reps))]
        finally:
            s.close()
        want = pending.get(timeout=3000)
    for k, (g, w) in enumerate(zip(got, want)):
        rc, n, eps, cnt = w
        assert rc == 0
        np.testing.assert_array_equal(g[0], n, err_msg=f"replica {k}")
        np.testing.assert_array_equal(np.asarray(g[1]).view(np.uint64), eps.view(np.uint64),
                                      err_msg=f"replica {k}")
        for f in ("rounds", "hops", "attempts", "P"):
            assert g[3][f] == cnt[f], (k, f)
        assert abs(g[3]["energy"] - cnt["energy"]) <= 1e-9 * max(1.0, abs(cnt["energy"])), k
