"""sigma(t) relaxation curves (Eq. 3) of the binary32 form against the
binary64 form at L=256 on thread-block clusters (the cluster-sized
workload): the paired differences of the window conductivities over the
replicas are consistent with zero (z per window), and both forms record
the same log-spaced time grid.
"""
import numpy as np
import pytest

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


def test_l256_sigma_binary32_matches_binary64(B):
    from paper_1407_5026_gb300 import sigma
    r = sigma.compare_forms_l256(B, 0, hops=40_000, R=8)
    assert r["clusters"]["fp32"] >= 2 and r["clusters"]["fp64"] >= 2
    assert r["windows"] >= 10
    assert np.all(np.diff(r["t"]) > 0)
    assert r["max_abs_z"] < 5.0 and r["rms_z"] < 2.0, r
    # the field drives current along +x at late times in both forms
    assert np.mean(r["sigma_fp64"][-5:]) > 0 and np.mean(r["sigma_fp32"][-5:]) > 0
