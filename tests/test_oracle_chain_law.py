"""Pins of the oracle chain's law against exact results.

* Detailed balance at E = 0 by exact enumeration (N=8 ring: 70 states;
  L=4 torus: 12870 states): the one-attempt kernel built from the oracle's
  proposal weights and dH satisfies pi_a K_ab = pi_b K_ba with
  pi ~ exp(-H/T), H from Eq. 1 evaluated by numpy.
* The oracle's actual trajectory visits states with the Boltzmann weights
  (attempt-weighted frequencies), which pins the random-number mapping, the
  tower sampling, the accept rule and the attempt accounting (p-1) M + q.
* Constant-acceptance closed forms of the parallel rejection section:
  <p> = 1/[1-(1-A)^M], <m> = 1/A, P(q = k) ~ (1-A)^(k-1).
* T -> infinity: a label accepts iff theta, with probability
  p_theta = sum_i sum_d p(d) n_i (1 - n_{i+d}) / N computed by brute force.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests import physics_ref as ref


def _states(N, k):
    out = []
    for occ in itertools.combinations(range(N), k):
        n = np.zeros(N, np.uint8)
        n[list(occ)] = 1
        out.append(n)
    return np.array(out)


def _kernel(c, states, quantised=True):
    """One-attempt transition matrix of the serial mixed algorithm."""
    Lx, Ly, N = c.Lx, c.Ly, c.N
    dxs, dys, Wi, w = c.vectors()
    pd = Wi.astype(np.float64) / 2.0 ** 32 if quantised else w / c.Z
    index = {s.tobytes(): a for a, s in enumerate(states)}
    K = np.zeros((len(states), len(states)))
    for a, n in enumerate(states):
        c.set_state(n)
        for i in range(N):
            if n[i] != 1:
                continue
            xi, yi = i % Lx, i // Lx
            for k in range(len(dxs)):
                j = ((yi + dys[k]) % Ly) * Lx + (xi + dxs[k]) % Lx
                if n[j] != 0:
                    continue
                dE = c.delta_e(i, j, int(dxs[k]))
                acc = min(1.0, math.exp(-dE / c.T))
                n2 = n.copy()
                n2[i], n2[j] = 0, 1
                K[a, index[n2.tobytes()]] += (1.0 / N) * pd[k] * acc
    K[np.diag_indices_from(K)] += 1.0 - K.sum(axis=1)
    return K


@pytest.mark.parametrize("geom", ["ring8", "torus4"])
def test_detailed_balance_exact_enumeration(geom):
    if geom == "ring8":
        c = oracle.Chain(8, 1, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.4, E=0.0, seed=4)
    else:
        c = oracle.Chain(4, 4, nu=0.5, W=1.0, xi=1.0, r_max=1, T=0.4, E=0.0, seed=4)
    n0, _, phi = c.state()
    states = _states(c.N, c.N // 2)
    assert len(states) == (70 if geom == "ring8" else 12870)
    G = ref.coupling_matrix(c.Lx, c.Ly)
    H = ref.interaction_energy_batch(states, phi, 0.5, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    for quantised in (True, False):
        K = _kernel(c, states, quantised)
        F = pi[:, None] * K
        scale = np.abs(F).max()
        assert np.abs(F - F.T).max() <= 1e-14 * scale
        np.testing.assert_allclose(pi @ K, pi, rtol=0, atol=1e-14)


def _visit_tv(c, n_hops, M, wrong_accounting=False):
    n0, _, phi = c.state()
    states = _states(c.N, c.N // 2)
    G = ref.coupling_matrix(c.Lx, c.Ly)
    H = ref.interaction_energy_batch(states, phi, 0.5, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    rc, log = c.run(n_hops, M, log=True)
    assert rc == oracle.ORC_OK
    # state before each hop as a bit code; a hop toggles bits i and j
    bit = 1 << np.arange(c.N, dtype=np.int64)
    code0 = int((n0.astype(np.int64) * bit).sum())
    toggles = (1 << log["i"].astype(np.int64)) | (1 << log["j"].astype(np.int64))
    codes = np.concatenate([[code0], code0 ^ np.bitwise_xor.accumulate(toggles)[:-1]])
    lookup = np.full(1 << c.N, -1, np.int64)
    lookup[(states.astype(np.int64) * bit).sum(axis=1)] = np.arange(len(states))
    idx = lookup[codes]
    assert (idx >= 0).all()
    m = (log["p"].astype(np.int64) - 1) * M + log["q"]
    if wrong_accounting:
        m = m + M          # the printed m = pM + q
    weight = np.bincount(idx, weights=m.astype(np.float64), minlength=len(states))
    f = weight / weight.sum()
    return 0.5 * np.abs(f - pi).sum()


@pytest.mark.parametrize("M", [1, 5])
def test_trajectory_visits_boltzmann_weights(M):
    c = oracle.Chain(8, 1, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.4, E=0.0, seed=4)
    # statistical TV at 8e5 hops is ~0.004 (it falls as 1/sqrt(hops)); the
    # printed accounting m = pM + q converges to a TV near 0.08
    tv = _visit_tv(c, 800_000, M)
    assert tv < 0.012, tv


def test_visit_test_detects_wrong_attempt_accounting():
    # the printed m = pM + q overweights states left after few rounds; with a
    # large M the bias shows in the same statistic that accepts the chain
    c = oracle.Chain(8, 1, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.4, E=0.0, seed=4)
    assert _visit_tv(c, 200_000, 64, wrong_accounting=True) > 0.03


@pytest.mark.parametrize("A0,M", [(0.5, 1), (0.5, 4), (0.01, 1), (0.01, 256),
                                  (3e-4, 256), (3e-4, 4096)])
def test_constant_acceptance_closed_forms(A0, M):
    c = oracle.Chain(16, nu=0.5, W=1.0, r_max=4, T=0.05, seed=9)
    c.set_toy(A0)
    hops = 3000 if A0 > 1e-3 else 1200
    rc, log = c.run(hops, M, log=True)
    assert rc == oracle.ORC_OK
    p = log["p"].astype(np.float64)
    m = (p - 1) * M + log["q"]
    s = 1.0 - (1.0 - A0) ** M
    p_mean, p_se = 1.0 / s, math.sqrt((1 - s) / s ** 2 / hops)
    assert abs(p.mean() - p_mean) <= 3.5 * p_se + 1e-12, (p.mean(), p_mean)
    m_mean, m_se = 1.0 / A0, math.sqrt((1 - A0) / A0 ** 2 / hops)
    assert abs(m.mean() - m_mean) <= 3.5 * m_se, (m.mean(), m_mean)
    # label of the executed hop: geometric truncated at M
    q = log["q"].astype(np.float64)
    k = np.arange(1, M + 1)
    pk = (1 - A0) ** (k - 1) * A0
    pk /= pk.sum()
    q_mean = float((k * pk).sum())
    q_se = math.sqrt(float(((k - q_mean) ** 2 * pk).sum()) / hops)
    assert abs(q.mean() - q_mean) <= 3.5 * q_se + 1e-12


def test_infinite_temperature_acceptance_is_theta():
    c = oracle.Chain(16, nu=0.5, W=1.0, r_max=4, T=1e30, E=0.0, seed=13)
    n, _, _ = c.state()
    dxs, dys, Wi, _ = c.vectors()
    L = 16
    p_theta = 0.0
    for i in range(L * L):
        if n[i] != 1:
            continue
        xi, yi = i % L, i // L
        for k in range(len(dxs)):
            j = ((yi + dys[k]) % L) * L + (xi + dxs[k]) % L
            if n[j] == 0:
                p_theta += float(Wi[k]) / 2.0 ** 32 / (L * L)
    K = 40_000
    acc = 0
    vec_count = np.zeros(len(dxs) + 1, np.int64)
    for k in range(K):
        lab = c.eval_label(k // 1000, k % 1000)
        acc += lab.accepted
        vec_count[lab.vec] += 1
        assert lab.accepted == lab.theta
    se = math.sqrt(p_theta * (1 - p_theta) / K)
    assert abs(acc / K - p_theta) <= 4 * se
    # sampled displacement frequencies follow the integer tower weights
    expct = Wi.astype(np.float64) / 2.0 ** 32 * K
    chi2 = float((((vec_count[:-1] - expct) ** 2) / expct).sum())
    assert chi2 < len(dxs) + 6 * math.sqrt(2 * len(dxs))
