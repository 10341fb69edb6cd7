"""The sigma(t) analysis arithmetic (Eq. 3 windows, the plateau sigma_0 and
Eq. 4's scaling variables) against hand-computed values and a family of
curves built to obey Eq. 4 exactly.  No GPU: the functions take traces."""
import numpy as np
import pytest

from paper_1407_5026_gb300 import sigma as S


def _trace(t, P):
    return {"time": np.asarray(t, dtype=np.float64), "P": np.asarray(P, dtype=np.int64)}


def test_windows_by_hand():
    # N E = 50; windows (5 - 0)/(50 * 1), (25 - 5)/(50 * 2), (85 - 25)/(50 * 4);
    # the zero-length window between the two points at t = 2 is dropped
    tr = _trace([1, 2, 2, 4, 8], [0, 5, 5, 25, 85])
    t, sig = S.sigma_windows(tr, 100, 0.5)
    np.testing.assert_allclose(t, [1.5, 3.0, 6.0])
    np.testing.assert_allclose(sig, [0.1, 0.2, 0.3])


def test_plateau_by_hand():
    tr = _trace([1, 2, 4, 8], [0, 5, 25, 85])
    assert S.sigma0_plateau(tr, 100, 0.5, 3.0) == pytest.approx(60 / 200)
    assert S.sigma0_plateau(tr, 100, 0.5, 2.0) == pytest.approx(80 / 300)
    assert np.isnan(S.sigma0_plateau(tr, 100, 0.5, 9.0))


def test_rescale_by_hand():
    x, y = S.rescale([1.5, 3.0, 6.0], [0.1, 0.2, 0.3], 0.3, 0.1)
    np.testing.assert_allclose(x, [0.0045, 0.009, 0.018])
    np.testing.assert_allclose(y, [1 / 3, 2 / 3, 1.0])


def test_mean_trace_keeps_common_points():
    a = _trace([1, 2, 4], [0, 2, 6])
    b = _trace([1, 2, 4, 8], [0, 4, 10, 30])
    m = S.mean_trace([a, b])
    np.testing.assert_allclose(m["time"], [1, 2, 4])
    np.testing.assert_allclose(m["P"], [0, 3, 8])


def test_curves_obeying_eq4_collapse_after_rescaling():
    # sigma(t, T) = sigma_0 f(t sigma_0 T^2) with f(x) = x / (1 + x) gives
    # P(t) = N E sigma_0 (t - ln(1 + x) / (sigma_0 T^2)); sampled on a fine
    # log grid, every temperature's rescaled windows lie on f, and the
    # plateau slope over the last decade approaches sigma_0
    N, E = 4096, 0.01
    for T, s0 in ((0.02, 3e-6), (0.05, 2e-4), (0.1, 4e-3)):
        tau = 1.0 / (s0 * T * T)
        t = np.logspace(np.log10(tau) - 3, np.log10(tau) + 4, 400)
        x_t = t * s0 * T * T
        P = N * E * s0 * (t - np.log1p(x_t) / (s0 * T * T))
        tr = {"time": t, "P": P}
        tm, sig = S.sigma_windows(tr, N, E)
        x, y = S.rescale(tm, sig, s0, T)
        np.testing.assert_allclose(y, x / (1 + x), rtol=2e-2, atol=1e-4)
        s0_est = S.sigma0_plateau(tr, N, E, t[-1] / 10)
        assert s0_est == pytest.approx(s0, rel=2e-3)
