"""The refresh entry point for callers that cannot allocate device memory.

cg_refresh_tc_noalloc serves code that may not call cudaMalloc itself (a host
program that owns the device allocator, a service with a fixed device
footprint).  It takes caller-owned device arrays and keeps all of its scratch
in one static device array.  These tests call it through the C ABI, with the
caller's arrays allocated by torch, and compare it with the handle-based
refresh (cg_refresh on a tensor-core batch) on the same state: the two run
the same kernels on the same inputs, so eps and the per-replica maximum error
must agree bit for bit, on two calls in a row.  eps is also compared with the
oracle's eps from its definition (phi + G (n - nu), below Eq. 2) within the
tensor-core refresh's tolerance.  The edges of the static scratch (the largest
accepted R at L = 128 and one more), a larger K split (L = 160) and a caller
stream other than the current one are covered too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 5e-5   # the tolerance of the tensor-core refresh tests


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def _device_inputs(sysm, R, L):
    import torch
    states = [sysm.state(k) for k in range(R)]
    occ = np.stack([np.packbits(s[0], bitorder="little").view(np.uint32) for s in states])
    phi = np.stack([s[2] for s in states])
    eps = np.stack([s[1] for s in states]).astype(np.float32)   # binary32 values, exact
    return (torch.from_numpy(np.ascontiguousarray(occ).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(phi)).cuda(),
            torch.from_numpy(np.ascontiguousarray(eps)).cuda(),
            torch.zeros(R, dtype=torch.float64, device="cuda"))


def _reps(L, R):
    return [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.03, E=0.01, seed=s, replica=s)
            for s in range(R)]


def _compare_with_handle(B, L, R, hops, calls, stream=None, oracle_check=()):
    """Runs `calls` rounds of (run, noalloc refresh, handle refresh) on R
    replicas of side L and checks the two refreshes agree bit for bit."""
    import torch
    sysm = B.System(_reps(L, R), precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_BF16X2)
    st = stream if stream is not None else torch.cuda.current_stream()
    try:
        for call in range(calls):
            sysm.run(hops * (call + 1), 1024)     # no refresh inside the run
            occ, phi, eps, err = _device_inputs(sysm, R, L)
            torch.cuda.synchronize()
            with torch.cuda.stream(st):
                rc = B.cg_refresh_tc_noalloc(L, R, 0.5, occ.data_ptr(), phi.data_ptr(),
                                             eps.data_ptr(), err.data_ptr(), st.cuda_stream)
            assert rc == B.CG_OK
            torch.cuda.synchronize()
            B.cg_refresh(sysm.h)                  # the handle's refresh, same state
            got = eps.cpu().numpy()
            errs = err.cpu().numpy()
            for k in range(R):
                n, want, phi_k, _ = sysm.state(k)
                np.testing.assert_array_equal(got[k].view(np.uint32),
                                              want.astype(np.float32).view(np.uint32),
                                              err_msg=f"call {call} replica {k}")
                obs = sysm.observables(k)
                assert errs[k] == obs["max_eps_err_last_refresh"], (call, k)
                if k in oracle_check:
                    import oracle
                    ch = oracle.Chain(L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.03, E=0.01,
                                      seed=k, replica=k)
                    ch.set_state(n, phi_k)
                    exact = ch.eps_scratch()
                    worst = float(np.abs(got[k].astype(np.float64) - exact).max())
                    assert worst <= TOL, (call, k, worst)
    finally:
        sysm.close()


def test_noalloc_refresh_matches_handle_refresh_on_two_calls(B):
    # bit for bit against the handle, and against the oracle's eps from its
    # definition on three replicas, on two calls in a row
    _compare_with_handle(B, 64, 24, 400, 2, oracle_check=(0, 11, 23))


def test_noalloc_refresh_at_the_largest_accepted_size(B):
    # L = 128: 48 replicas use 26.8 MB of the 32 MiB array
    _compare_with_handle(B, 128, 48, 200, 1, oracle_check=(47,))


def test_noalloc_refresh_with_a_larger_k_split_on_another_stream(B):
    # L = 160 splits the contraction's K range 10 ways (8 below); the caller's
    # stream is not the current one
    import torch
    _compare_with_handle(B, 160, 16, 200, 2, stream=torch.cuda.Stream())


def test_noalloc_refresh_refuses_sizes_beyond_its_scratch(B):
    import torch
    for L, R in ((128, 49), (128, 512), (192, 1)):
        N = L * L
        occ = torch.zeros(R * N // 32, dtype=torch.int32, device="cuda")
        phi = torch.zeros(R * N, dtype=torch.float64, device="cuda")
        eps = torch.zeros(R * N, dtype=torch.float32, device="cuda")
        with pytest.raises(B.CgError) as ei:
            B.cg_refresh_tc_noalloc(L, R, 0.5, occ.data_ptr(), phi.data_ptr(), eps.data_ptr())
        assert ei.value.code == B.CG_EINVAL
        assert "static maximum" in str(ei.value)
