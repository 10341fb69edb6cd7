"""Pins of the oracle's random-site Coulomb glass (reading R16).

* Positions equal the Philox definition; the partner lists, 1/r and the
  minimum-image dx of every pair equal a numpy brute force over all pairs.
* The integer tower weights are symmetric (W_ij = W_ji), so a proposal and
  its reverse have the same probability; Gamma = N Zmax.
* eps and dH equal numpy evaluations of Eq. 1 with the minimum-image
  distances of the random positions (the field term uses the real dx).
* Detailed balance of the one-attempt kernel by exact enumeration of every
  half-filled state of 16 random sites, with energies from numpy.
* The oracle's labels from a fixed state hit each target with the kernel
  row's probability (chi-square); incremental eps and energy after a run
  equal their values from scratch.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads
from tests import physics_ref as ref


def _geometry(c):
    L = c.Lx
    x, y = c.positions()
    dx = x[None, :] - x[:, None]
    dy = y[None, :] - y[:, None]
    dx = np.where(dx > 0.5 * L, dx - L, np.where(dx < -0.5 * L, dx + L, dx))
    dy = np.where(dy > 0.5 * L, dy - L, np.where(dy < -0.5 * L, dy + L, dy))
    r = np.sqrt(dx * dx + dy * dy)
    with np.errstate(divide="ignore"):
        G = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    return dx, r, G


def test_positions_follow_the_philox_definition():
    c = oracle.Chain(8, r_max=2, seed=11, replica=3, random_sites=True)
    x, y = c.positions()
    for s in (0, 1, 17, 63):
        w = oracle.philox([s, 3, 0xFFFFFFFF, 3], [11, 0])
        assert x[s] == 8.0 * ((float(w[0]) + 0.5) * 2.0 ** -32)
        assert y[s] == 8.0 * ((float(w[1]) + 0.5) * 2.0 ** -32)
    assert np.all((x > 0) & (x < 8) & (y > 0) & (y < 8))


@pytest.mark.parametrize("L,r_max", [(8, 2), (10, 3)])
def test_partner_lists_equal_a_brute_force(L, r_max):
    c = oracle.Chain(L, r_max=r_max, xi=1.3, seed=5, random_sites=True)
    dx, r, G = _geometry(c)
    off, j, C, g, pdx = c.pairs()
    N = c.N
    for s in range(N):
        want = [t for t in range(N) if t != s and r[s, t] <= r_max]
        got = j[off[s]:off[s + 1]].tolist()
        assert got == want
        np.testing.assert_array_equal(g[off[s]:off[s + 1]], G[s, want])
        np.testing.assert_array_equal(pdx[off[s]:off[s + 1]], dx[s, want])
    # integer weights: symmetric, and their per-site sums at most 2^32
    Wm = {}
    for s in range(N):
        for m in range(off[s], off[s + 1]):
            Wm[(s, int(j[m]))] = int(C[m]) - (int(C[m - 1]) if m > off[s] else 0)
    for (a, b), w in Wm.items():
        assert Wm[(b, a)] == w
    assert all(int(C[off[s + 1] - 1]) <= 2 ** 32 for s in range(N) if off[s + 1] > off[s])
    assert c.Gamma == N * c.Zmax


@pytest.mark.parametrize("E", [0.0, 0.07])
def test_eps_and_delta_e_equal_eq1(E):
    L = 8
    N = L * L
    c = oracle.Chain(L, r_max=2, T=0.1, E=E, seed=2, random_sites=True)
    dx, r, G = _geometry(c)
    rng = np.random.default_rng(4)
    n = workloads.random_occupation(N, N // 2, seed=7)
    phi = workloads.random_phi(N, 1.0, seed=8)
    c.set_state(n, phi)
    assert np.abs(c.state()[1] - ref.site_energies(n, phi, 0.5, G)).max() <= 1e-12
    H0 = ref.interaction_energy(n, phi, 0.5, G)
    _, eps, _ = c.state()
    off, j, C, g, pdx = c.pairs()
    checked = 0
    for _ in range(200):
        i = int(rng.choice(np.nonzero(n)[0]))
        if off[i + 1] == off[i]:
            continue
        m = int(rng.integers(off[i], off[i + 1]))
        jj = int(j[m])
        if n[jj]:
            continue
        dH = ((eps[jj] - eps[i]) - g[m]) - E * pdx[m]
        n2 = n.copy()
        n2[i], n2[jj] = 0, 1
        want = (ref.interaction_energy(n2, phi, 0.5, G) - H0) - E * dx[i, jj]
        assert abs(dH - want) <= 1e-12 * (1 + abs(H0) / N)
        checked += 1
    assert checked > 50


def _states(N, k):
    out = []
    for occ in itertools.combinations(range(N), k):
        n = np.zeros(N, np.uint8)
        n[list(occ)] = 1
        out.append(n)
    return np.array(out)


def _kernel_row(c, n, index, H_of, E):
    """One attempt from n with the oracle's integer weights and energies
    from numpy: {target: probability}."""
    N = c.N
    off, j, C, g, pdx = c.pairs()
    row = {}
    H0 = H_of(n)
    for i in np.nonzero(n)[0]:
        for m in range(off[i], off[i + 1]):
            jj = int(j[m])
            if n[jj]:
                continue
            W = int(C[m]) - (int(C[m - 1]) if m > off[i] else 0)
            n2 = n.copy()
            n2[i], n2[jj] = 0, 1
            dH = H_of(n2) - H0 - E * pdx[m]
            acc = min(1.0, math.exp(-dH / c.T))
            b = index(n2)
            row[b] = row.get(b, 0.0) + (1.0 / N) * (W * 2.0 ** -32) * acc
    return row


def test_detailed_balance_on_random_sites():
    L = 4
    N = L * L
    c = oracle.Chain(L, r_max=1, xi=1.0, T=0.4, E=0.0, seed=9, random_sites=True)
    _, _, phi = c.state()
    _, _, G = _geometry(c)
    states = _states(N, N // 2)
    H = ref.interaction_energy_batch(states, phi, 0.5, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    lookup = {s.tobytes(): a for a, s in enumerate(states)}
    Hmap = dict(zip((s.tobytes() for s in states), H))
    K = np.zeros((len(states), len(states)))
    for a, n in enumerate(states):
        for b, v in _kernel_row(c, n, lambda s: lookup[s.tobytes()],
                                lambda s: Hmap[s.tobytes()], 0.0).items():
            K[a, b] += v
    K[np.diag_indices_from(K)] += 1.0 - K.sum(axis=1)
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    assert (K > 0).sum() > 3 * len(states)


def test_labels_follow_the_kernel_row():
    L = 6
    N = L * L
    c = oracle.Chain(L, r_max=2, xi=1.0, T=0.5, E=0.05, seed=12, random_sites=True)
    n, _, phi = c.state()
    _, _, G = _geometry(c)
    row = _kernel_row(c, n, lambda s: s.tobytes(),
                      lambda s: ref.interaction_energy(s, phi, 0.5, G), c.E)
    n_labels = 300_000
    counts = {}
    for t in range(n_labels):
        lab = c.eval_label(t // 64, t % 64)
        if lab.accepted:
            n2 = n.copy()
            n2[lab.i], n2[lab.j] = 0, 1
            b = n2.tobytes()
            counts[b] = counts.get(b, 0) + 1
    assert set(counts) <= set(row)
    chi2, dof = 0.0, 0
    for b, pb in row.items():
        e = pb * n_labels
        if e >= 5:
            chi2 += (counts.get(b, 0) - e) ** 2 / e
            dof += 1
    assert dof >= 20
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_random_site_run_keeps_eps_and_energy():
    L = 10
    c = oracle.Chain(L, r_max=2, T=0.2, E=0.03, seed=6, random_sites=True)
    n0 = c.state()[0]
    x, _ = c.positions()
    P0 = float((n0 * x).sum())            # the initial dipole of the real positions
    rc, log = c.run(2000, 128, log=True)
    assert rc == oracle.ORC_OK
    n, eps, phi = c.state()
    assert np.abs(eps - c.eps_scratch()).max() <= 1e-11
    _, _, G = _geometry(c)
    H = ref.interaction_energy(n, phi, 0.5, G)
    # the energy counter is H - E P with the unwrapped dipole P = P0 + the
    # hops' minimum-image dx (as on the lattice)
    off, j, C, g, pdx = c.pairs()
    P = P0
    for e in log:
        m = off[e["i"]] + list(j[off[e["i"]]:off[e["i"] + 1]]).index(e["j"])
        P += pdx[m]
    assert abs(c.counters()["energy"] - (H - c.E * P)) <= 1e-9 * max(1.0, abs(H))
    assert c.counters()["P"] == 0
