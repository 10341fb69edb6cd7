"""The refresh entry point for callers that cannot allocate device memory.

cg_refresh_tc_noalloc serves code that may not call cudaMalloc itself (a host
program that owns the device allocator, a service with a fixed device
footprint).  It takes caller-owned device arrays and keeps all of its scratch
in one static device array.  These tests call it through the C ABI, with the
caller's arrays allocated by torch, and compare its eps and per-replica
maximum error with the handle-based refresh (cg_refresh on a tensor-core
batch) on the same state, on two calls in a row.  Sizes beyond the static
scratch are refused with a clear error.
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


def test_noalloc_refresh_matches_handle_refresh_on_two_calls(B):
    import torch
    L, R = 64, 24
    reps = [dict(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.03, E=0.01, seed=s, replica=s)
            for s in range(R)]
    sysm = B.System(reps, precision=B.CG_FP32, refresh_kind=B.CG_REFRESH_BF16X2)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for call in range(2):
            sysm.run(400 * (call + 1), 1024)      # no refresh inside the run
            occ, phi, eps, err = _device_inputs(sysm, R, L)
            torch.cuda.synchronize()
            rc = B.cg_refresh_tc_noalloc(L, R, 0.5, occ.data_ptr(), phi.data_ptr(),
                                         eps.data_ptr(), err.data_ptr(), stream)
            assert rc == B.CG_OK
            B.cg_refresh(sysm.h)                  # the handle's refresh, same state
            got = eps.cpu().numpy().astype(np.float64)
            errs = err.cpu().numpy()
            for k in range(R):
                want = sysm.state(k)[1]
                assert np.abs(got[k] - want).max() <= TOL, (call, k)
                obs = sysm.observables(k)
                assert abs(errs[k] - obs["max_eps_err_last_refresh"]) <= TOL, (call, k)
    finally:
        sysm.close()


def test_noalloc_refresh_refuses_sizes_beyond_its_scratch(B):
    import torch
    L, R = 128, 512
    N = L * L
    occ = torch.zeros(R * N // 32, dtype=torch.int32, device="cuda")
    phi = torch.zeros(R * N, dtype=torch.float64, device="cuda")
    eps = torch.zeros(R * N, dtype=torch.float32, device="cuda")
    with pytest.raises(B.CgError) as ei:
        B.cg_refresh_tc_noalloc(L, R, 0.5, occ.data_ptr(), phi.data_ptr(), eps.data_ptr())
    assert ei.value.code == B.CG_EINVAL
    assert "static maximum" in str(ei.value)
