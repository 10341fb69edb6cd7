"""The binary32 form against the binary64 form at the headline configuration.

Workload: L = 128 (N = 16384), nu = 1/2, phi ~ U[-1, 1] (W = 2), xi = 1,
r_max = 8, T = 0.01, E = 0.005 along x, M = 4096; binary32 eps refreshed every
1024 hops.  Criterion: over 64 disorder samples the binary32 form's
observables lie within two standard errors of the binary64 form's, and its eps
stays within 1e-4 of the definition below Eq. 2.

Procedure (fixed seeds 0..63):

1. 64 binary64 replicas relax 40960 hops from their random start.
2. Each relaxed state (occupation, eps, phi, counters) is written into a
   binary32 handle of the same replicas, with its round counter moved by
   2^40.  From there the two forms draw disjoint Philox counters: the same
   disorder and start, independent trajectories (the chain's law does not
   depend on which random numbers a label draws).
3. Both forms run 65536 more hops.  Per sample: the interaction energy per site
   of the final configuration (H of Eq. 1 without the field term, from
   scratch), the dipole change P1 - P0 and the acceptance over the run.  The
   paired differences binary32 - binary64 over the 64 samples give
   z = mean / SE, with |z| < 2 required for each observable.
4. eps of the binary32 form: the largest error any refresh saw, and eps at
   the end against phi + G (n - nu) from scratch, both <= 1e-4.
"""
import math

import numpy as np
import pytest

from tests import physics_ref as ref

pytestmark = pytest.mark.gpu

L, NU, W, XI, RMAX, T, E = 128, 0.5, 2.0, 1.0, 8, 0.01, 0.005
SAMPLES, RELAX, HOPS, M = 64, 40960, 65536, 4096
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


def _observables(sysm, k, c0):
    n, eps, phi, c = sysm.state(k)
    exact = ref.site_energies_fft(n, phi, NU, L)
    h_int = float(phi @ n + 0.5 * (n - NU) @ (exact - phi))
    dh, da = c["hops"] - c0["hops"], c["attempts"] - c0["attempts"]
    return [h_int / L ** 2, float(c["P"] - c0["P"]), dh / da], float(np.abs(eps - exact).max())


def test_binary32_within_two_standard_errors_of_binary64_at_L128_T001(B):
    reps = [dict(L=L, nu=NU, W=W, xi=XI, r_max=RMAX, T=T, E=E, seed=s, replica=s)
            for s in range(SAMPLES)]
    s64 = B.System(reps, precision=B.CG_FP64)
    s32 = B.System(reps, precision=B.CG_FP32, refresh_every=1024)
    try:
        assert s64.run(RELAX, M) == B.CG_OK
        start = []
        for k in range(SAMPLES):
            n, eps, phi, c = s64.state(k)
            start.append(c)
            c32 = dict(c)
            c32["rounds"] = c["rounds"] + ROUND_SHIFT
            B.cg_write_state(s32.h, k, n, eps=eps, phi=phi, counters=c32)
        assert s64.run(HOPS, M) == B.CG_OK
        assert s32.run(HOPS, M) == B.CG_OK
        v64, v32, eps_err = [], [], 0.0
        for k in range(SAMPLES):
            v, _ = _observables(s64, k, start[k])
            v64.append(v)
            v, err = _observables(s32, k, start[k])
            v32.append(v)
            eps_err = max(eps_err, err)
            assert s32.observables(k)["max_eps_err_last_refresh"] <= 1e-4
        d = np.array(v32) - np.array(v64)
        report = {}
        for col, name in enumerate(("E/N", "P", "A")):
            se = d[:, col].std(ddof=1) / math.sqrt(SAMPLES)
            z = d[:, col].mean() / se
            report[name] = (float(d[:, col].mean()), float(se), float(z))
        print("binary32 - binary64 (mean, SE, z):", report, "eps error", eps_err)
        for name, (_, se, z) in report.items():
            assert se > 0, name                 # independent trajectories, not copies
            assert abs(z) < 2.0, (name, report)
        assert eps_err <= 1e-4, eps_err
    finally:
        s32.close()
        s64.close()
