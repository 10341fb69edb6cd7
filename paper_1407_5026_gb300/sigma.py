"""Conductivity relaxation sigma(t) from the library's dipole traces.

Analysis above the C ABI, not a step of the chain: the chain runs in libcg's
kernels, which record a log-spaced trace of the dipole moment P (cg_set_trace,
cg_read_trace); this module turns traces into the paper's observables.

* Eq. 3: sigma(t) = (1 / N E) dP/dt, estimated over the window between
  consecutive trace points (sigma_windows).
* sigma_0: the stationary conductivity, the late-time plateau of sigma(t),
  estimated as the mean slope of P over the last windows (sigma0_plateau).
* Eq. 4 (section "Results for the lattice model in two dimensions"): the
  relaxation follows sigma(t, T) = sigma_0 f(t sigma_0 T^2), so sigma / sigma_0
  against t sigma_0 T^2 should fall on one curve for all T (rescale).

The two drivers run the library on the synthetic configurations of the
relaxation experiment: relaxation_curves (L = 64, one disorder set per
temperature) and compare_forms_l256 (binary32 against binary64 on clusters).
Only the arithmetic of the rescaling is pinned (tests/test_sigma_analysis.py);
that the curves of different T collapse is the paper's finding, whose data
are not available here, so the collapse itself is unpinned.
"""
from __future__ import annotations

import numpy as np


def sigma_windows(trace, N, E):
    """Eq. 3 over the windows between consecutive trace points: returns
    (t_mid, sigma) with sigma_k = (P_{k+1} - P_k) / (N E (t_{k+1} - t_k)) and
    t_mid the window's midpoint, for the windows of positive length (the
    time each point recorded: attempts / Gamma, or the stochastic clock)."""
    t = np.asarray(trace["time"], dtype=np.float64)
    P = np.asarray(trace["P"], dtype=np.float64)
    dt = np.diff(t)
    keep = dt > 0
    t_mid = 0.5 * (t[1:] + t[:-1])[keep]
    return t_mid, (np.diff(P)[keep] / dt[keep]) / (N * E)


def sigma0_plateau(trace, N, E, t_from):
    """sigma_0 as the slope of P between the first trace point at or after
    t_from and the last point: (P_last - P_a) / (N E (t_last - t_a)), the
    length-weighted mean of the windows in that range.  NaN when fewer than
    two points lie in the range."""
    t = np.asarray(trace["time"], dtype=np.float64)
    P = np.asarray(trace["P"], dtype=np.float64)
    idx = np.nonzero(t >= t_from)[0]
    if len(idx) < 2 or t[-1] <= t[idx[0]]:
        return float("nan")
    a = idx[0]
    return float((P[-1] - P[a]) / (N * E * (t[-1] - t[a])))


def rescale(t, sigma, sigma0, T):
    """Eq. 4's scaling variables: (t sigma_0 T^2, sigma / sigma_0)."""
    t = np.asarray(t, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    return t * sigma0 * T * T, sigma / sigma0


def mean_trace(traces):
    """Points common to all traces (same log-spaced grid): the replicas'
    mean P at each point and the mean time."""
    K = min(len(tr["time"]) for tr in traces)
    t = np.mean([np.asarray(tr["time"][:K], dtype=np.float64) for tr in traces], axis=0)
    P = np.mean([np.asarray(tr["P"][:K], dtype=np.float64) for tr in traces], axis=0)
    return {"time": t, "P": P}


def relaxation_curves(B, device=0, temperatures=(0.02, 0.05, 0.1), seeds=range(8),
                      hops=1_000_000, M=4096, precision=None, points_per_decade=4.0,
                      first_time=1.0, plateau_decades=1.0):
    """sigma(t) of the L = 64 relaxation configuration (nu = 1/2, W = 1, xi = 1,
    r_max = 6, E = 0.01 along x) from the random start: every (temperature,
    disorder seed) chain in one handle (one persistent launch), the disorder
    of seed s the same at every T.  Per T: the replica-mean trace, its Eq. 3
    windows, sigma_0 as the slope of P over the last `plateau_decades`
    decades of the run's time, the acceptance, and the Eq. 4 variables
    (x, y) = (t sigma_0 T^2, sigma / sigma_0)."""
    from paper_1407_5026_gb300 import workloads as W
    prec = B.CG_FP64 if precision is None else precision
    seeds = list(seeds)
    base = W.l64_fp64(T=temperatures[0], seed=0, hops=hops).replicas[0].as_dict()
    reps = [dict(base, T=T, seed=s, replica=s) for T in temperatures for s in seeds]
    s = B.System(reps, precision=prec, refresh_every=1024 if prec == B.CG_FP32 else 0,
                 device=device)
    try:
        cap = 256
        B.cg_set_trace(s.h, first_time=first_time, points_per_decade=points_per_decade,
                       capacity=cap)
        rc = s.run(hops, M)
        assert rc == B.CG_OK, rc
        tr = [B.cg_read_trace(s.h, k, cap) for k in range(len(reps))]
        acc = [s.observables(k)["acceptance"] for k in range(len(reps))]
    finally:
        s.close()
    N, E = base["L"] ** 2, base["E"]
    out = {}
    for ti, T in enumerate(temperatures):
        sl = slice(ti * len(seeds), (ti + 1) * len(seeds))
        m = mean_trace(tr[sl])
        t_mid, sig = sigma_windows(m, N, E)
        t_end = float(m["time"][-1])
        s0 = sigma0_plateau(m, N, E, t_end / 10 ** plateau_decades)
        x, y = rescale(t_mid, sig, s0, T)
        out[T] = {"t": t_mid.tolist(), "sigma": sig.tolist(), "sigma0": s0,
                  "t_end": t_end, "acceptance": float(np.mean(acc[sl])),
                  "replicas": len(seeds), "hops": hops, "x": x.tolist(), "y": y.tolist()}
    return out


def compare_forms_l256(B, device=0, hops=200_000, R=16, points_per_decade=5.0,
                       first_time=1e-3):
    """sigma(t) curves (Eq. 3) of the L=256 configuration in the binary32 form
    (cluster kernel, refresh every 4096 hops) against the binary64 form,
    same seeds: each replica's trace records P at the log-spaced times t_k
    (point k of both runs belongs to t_k), so the window
    sigma_k = (P_{k+1} - P_k) / (N E (t_{k+1} - t_k)) pairs across the forms
    and the paired differences over the replicas give one z per window."""
    from paper_1407_5026_gb300 import workloads as W
    wl = W.l256(R=R)
    reps = [r.as_dict() for r in wl.replicas]
    N, E = 256 * 256, wl.replicas[0].E
    cap = 128
    sig, tmid, shape = {}, {}, {}
    for name, prec in (("fp32", B.CG_FP32), ("fp64", B.CG_FP64)):
        s = B.System(reps, precision=prec, device=device,
                     refresh_every=wl.refresh_every if prec == B.CG_FP32 else 0)
        try:
            B.cg_set_trace(s.h, first_time=first_time, points_per_decade=points_per_decade,
                           capacity=cap)
            assert s.run(hops, wl.M) == B.CG_OK
            tr = [B.cg_read_trace(s.h, k, cap) for k in range(R)]
            shape[name] = B.cg_group_shape(s.h, 0)["cluster"]
        finally:
            s.close()
        K = min(len(t) for t in tr)
        t = np.array([x["time"][:K] for x in tr], dtype=np.float64)
        Pk = np.array([x["P"][:K] for x in tr], dtype=np.float64)
        sig[name] = np.diff(Pk, axis=1) / (N * E * np.diff(t, axis=1))
        tmid[name] = 0.5 * (t[:, 1:] + t[:, :-1]).mean(axis=0)
    K = min(sig["fp32"].shape[1], sig["fp64"].shape[1])
    d = sig["fp32"][:, :K] - sig["fp64"][:, :K]
    se = d.std(axis=0, ddof=1) / np.sqrt(R)
    z = np.where(se > 0, d.mean(axis=0) / np.where(se > 0, se, 1.0), 0.0)
    return {"replicas": R, "hops_per_replica": hops, "windows": int(K),
            "clusters": shape, "t": tmid["fp64"][:K].round(6).tolist(),
            "sigma_fp32": sig["fp32"][:, :K].mean(axis=0).round(6).tolist(),
            "sigma_fp64": sig["fp64"][:, :K].mean(axis=0).round(6).tolist(),
            "max_abs_z": float(np.abs(z).max()), "rms_z": float(np.sqrt((z ** 2).mean()))}
