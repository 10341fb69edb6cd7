"""Pins of the oracle's two-electron hops (the multi-electron hops the paper
names as a straightforward extension; reading R15).

* dH of a pair move equals H(after) - H(before) - E (dx1 + dx2), H from
  Eq. 1 evaluated by numpy with its own coupling matrix, for random states
  and every kind of pair (neighbouring electrons, shared neighbourhoods).
* Detailed balance by exact enumeration on a 4 x 4 torus with three
  electrons: the one-attempt kernel of single and pair proposals (pair
  probability T_p 2^-32, offset uniform on the square [-R, R]^2 and kept
  inside the disk, reverse offset e' = e + d2 - d1 inside the disk) satisfies
  pi_a K_ab = pi_b K_ba with pi ~ exp(-H/T).  Dropping the reverse-offset
  condition breaks it, so the test sees that condition.
* The oracle's own labels, evaluated for many (round, label) counters from a
  fixed state, hit each target state with the probability the kernel row
  gives: this pins the second Philox block, the offset and tower draws, the
  pair theta and the acceptance against the definition above.
* The oracle's trajectory visits states with the Boltzmann weights
  (attempt-weighted), and its incremental eps, energy and dipole after a run
  with pair hops equal their values from scratch.
* p2 = 0 reproduces the single-hop chain exactly; Gamma = N Z / (1 - T_p 2^-32).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads
from tests import physics_ref as ref


def _pair_moves(c, n, R, require_reverse=True):
    """Every pair proposal (i, v1, ex, ey, v2) from occupation n with its
    probability given a pair label, and the resulting move when it passes
    theta: yields (prob, i, j, k, l, dx1, dx2)."""
    Lx, Ly, N = c.Lx, c.Ly, c.N
    dxs, dys, Wi, _ = c.vectors()
    pd = Wi.astype(np.float64) / 2.0 ** 32
    W = 2 * R + 1
    for i in np.nonzero(n)[0]:
        xi, yi = i % Lx, i // Lx
        for v1 in range(len(dxs)):
            j = ((yi + dys[v1]) % Ly) * Lx + (xi + dxs[v1]) % Lx
            if n[j]:
                continue
            for ex in range(-R, R + 1):
                for ey in range(-R, R + 1):
                    if not 0 < ex * ex + ey * ey <= R * R:
                        continue
                    xk, yk = (xi + ex) % Lx, (yi + ey) % Ly
                    k = yk * Lx + xk
                    if not n[k]:
                        continue
                    for v2 in range(len(dxs)):
                        l = ((yk + dys[v2]) % Ly) * Lx + (xk + dxs[v2]) % Lx
                        if n[l]:
                            continue
                        fx, fy = ex + dxs[v2] - dxs[v1], ey + dys[v2] - dys[v1]
                        if not 0 < fx * fx + fy * fy:
                            continue
                        if require_reverse and fx * fx + fy * fy > R * R:
                            continue
                        yield ((1.0 / N) * pd[v1] * pd[v2] / (W * W),
                               int(i), int(j), int(k), int(l), int(dxs[v1]), int(dxs[v2]))


def _kernel_row(c, n, R, p2q, index, require_reverse=True):
    """One attempt from n: single proposals with probability 1 - p2q, pairs
    with p2q (p2q = T_p 2^-32)."""
    Lx, Ly, N = c.Lx, c.Ly, c.N
    dxs, dys, Wi, _ = c.vectors()
    pd = Wi.astype(np.float64) / 2.0 ** 32
    row = {}
    c.set_state(n)
    for i in np.nonzero(n)[0]:
        xi, yi = i % Lx, i // Lx
        for v in range(len(dxs)):
            j = ((yi + dys[v]) % Ly) * Lx + (xi + dxs[v]) % Lx
            if n[j]:
                continue
            acc = min(1.0, math.exp(-c.delta_e(i, j, int(dxs[v])) / c.T))
            n2 = n.copy()
            n2[i], n2[j] = 0, 1
            b = index[n2.tobytes()]
            row[b] = row.get(b, 0.0) + (1.0 - p2q) * (1.0 / N) * pd[v] * acc
    for prob, i, j, k, l, dx1, dx2 in _pair_moves(c, n, R, require_reverse):
        acc = min(1.0, math.exp(-c.delta_e_pair(i, j, k, l, dx1, dx2) / c.T))
        n2 = n.copy()
        n2[i], n2[j], n2[k], n2[l] = 0, 1, 0, 1
        b = index[n2.tobytes()]
        row[b] = row.get(b, 0.0) + p2q * prob * acc
    return row


def _states(N, k):
    out = []
    for occ in itertools.combinations(range(N), k):
        n = np.zeros(N, np.uint8)
        n[list(occ)] = 1
        out.append(n)
    return np.array(out)


def _small_chain(**kw):
    p = dict(nu=3 / 16, W=1.0, xi=1.0, r_max=1, T=0.5, E=0.0, seed=4, pair_frac=0.4, pair_rmax=1)
    p.update(kw)
    return oracle.Chain(4, 4, **p)


@pytest.mark.parametrize("E", [0.0, 0.07])
def test_pair_delta_e_equals_hamiltonian_difference(E):
    L = 6
    N = L * L
    c = oracle.Chain(L, L, r_max=2, T=0.1, E=E, seed=2, pair_frac=0.3, pair_rmax=2)
    G = ref.coupling_matrix(L, L)
    rng = np.random.default_rng(8)
    checked = 0
    for trial in range(3):
        n = workloads.random_occupation(N, N // 2, seed=40 + trial)
        phi = workloads.random_phi(N, 1.0, seed=50 + trial)
        c.set_state(n, phi)
        H0 = ref.interaction_energy(n, phi, 0.5, G)
        moves = list(_pair_moves(c, n, 2))
        for m in rng.choice(len(moves), 80, replace=False):
            _, i, j, k, l, dx1, dx2 = moves[m]
            n2 = n.copy()
            n2[i], n2[j], n2[k], n2[l] = 0, 1, 0, 1
            want = (ref.interaction_energy(n2, phi, 0.5, G) - H0) - E * (dx1 + dx2)
            got = c.delta_e_pair(i, j, k, l, dx1, dx2)
            assert abs(got - want) <= 1e-12 * (1 + abs(H0) / N), (i, j, k, l)
            checked += 1
    assert checked == 240


def test_pair_detailed_balance_exact_enumeration():
    c = _small_chain()
    _, _, phi = c.state()
    states = _states(c.N, 3)
    index = {s.tobytes(): a for a, s in enumerate(states)}
    G = ref.coupling_matrix(4, 4)
    H = ref.interaction_energy_batch(states, phi, 3 / 16, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    p2q = c.pair_threshold * 2.0 ** -32
    assert c.pair_threshold == math.floor(0.4 * 2.0 ** 32)

    def kernel(require_reverse):
        K = np.zeros((len(states), len(states)))
        for a, n in enumerate(states):
            for b, v in _kernel_row(c, n, 1, p2q, index, require_reverse).items():
                K[a, b] += v
        K[np.diag_indices_from(K)] += 1.0 - K.sum(axis=1)
        return K

    K = kernel(True)
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    # pair moves are present and carry weight
    assert (K > 0).sum() > len(states) * 10
    # without the reverse-offset condition the proposal is not symmetric
    K_bad = kernel(False)
    F_bad = pi[:, None] * K_bad
    assert np.abs(F_bad - F_bad.T).max() > 1e-6 * np.abs(F_bad).max()


def test_oracle_labels_follow_the_kernel_row():
    c = _small_chain(T=0.6)
    states = _states(c.N, 3)
    index = {s.tobytes(): a for a, s in enumerate(states)}
    # electrons at (0, 0), (1, 0) (neighbours: pair moves exist) and (2, 2)
    n = np.zeros(16, np.uint8)
    n[[0, 1, 10]] = 1
    c.set_state(n)
    p2q = c.pair_threshold * 2.0 ** -32
    row = _kernel_row(c, n, 1, p2q, index)
    n_labels = 400_000
    counts = {}
    pairs = 0
    for t in range(n_labels):
        lab = c.eval_label(t // 64, t % 64)
        pairs += lab.pair
        if lab.accepted:
            n2 = n.copy()
            n2[lab.i], n2[lab.j] = 0, 1
            if lab.pair:
                n2[lab.k], n2[lab.l] = 0, 1
            b = index[n2.tobytes()]
            counts[b] = counts.get(b, 0) + 1
    # every reached state is one the kernel allows, and the frequencies match
    assert set(counts) <= set(row)
    assert abs(pairs / n_labels - p2q) < 5 * math.sqrt(p2q * (1 - p2q) / n_labels)
    chi2, dof = 0.0, 0
    for b, pb in row.items():
        e = pb * n_labels
        if e >= 20:
            chi2 += (counts.get(b, 0) - e) ** 2 / e
            dof += 1
    assert dof >= 10
    # chi-square with dof degrees of freedom: mean dof, sd sqrt(2 dof)
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)
    # pair targets (four sites changed) are reached
    four = [b for b in counts if np.abs(states[b].astype(int) - n).sum() == 4]
    assert sum(counts[b] for b in four) > 100


def test_pair_trajectory_visits_boltzmann_weights():
    c = _small_chain(T=0.5)
    n0, _, phi = c.state()
    states = _states(c.N, 3)
    G = ref.coupling_matrix(4, 4)
    H = ref.interaction_energy_batch(states, phi, 3 / 16, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    M = 4
    rc, log = c.run(300_000, M, log=True)
    assert rc == oracle.ORC_OK
    pair = log["k"] != 0xFFFFFFFF
    assert pair.sum() > 300
    bit = 1 << np.arange(c.N, dtype=np.int64)
    code0 = int((n0.astype(np.int64) * bit).sum())
    toggles = (1 << log["i"].astype(np.int64)) | (1 << log["j"].astype(np.int64))
    toggles = toggles | np.where(pair, (1 << log["k"].astype(np.int64)) |
                                 (1 << log["l"].astype(np.int64)), 0)
    codes = np.concatenate([[code0], code0 ^ np.bitwise_xor.accumulate(toggles)[:-1]])
    lookup = np.full(1 << c.N, -1, np.int64)
    lookup[(states.astype(np.int64) * bit).sum(axis=1)] = np.arange(len(states))
    idx = lookup[codes]
    assert (idx >= 0).all()
    m = (log["p"].astype(np.int64) - 1) * M + log["q"]
    f = np.bincount(idx, weights=m.astype(np.float64), minlength=len(states))
    f /= f.sum()
    tv = 0.5 * np.abs(f - pi).sum()
    # 560 states: the statistical TV at 3e5 hops is ~0.01
    assert tv < 0.025, tv


def test_pair_run_keeps_eps_energy_and_dipole():
    L = 12
    c = oracle.Chain(L, L, r_max=3, T=0.3, E=0.02, seed=9, pair_frac=0.25, pair_rmax=3)
    n0, _, phi = c.state()
    P0 = c.counters()["P"]
    rc, log = c.run(3000, 128, log=True)
    assert rc == oracle.ORC_OK
    pair = log["k"] != 0xFFFFFFFF
    assert pair.sum() > 20
    n, eps, _ = c.state()
    assert np.abs(eps - c.eps_scratch()).max() <= 1e-11
    cnt = c.counters()
    assert cnt["P"] - P0 == int(log["dx"].sum() + log["dx2"].sum())
    G = ref.coupling_matrix(L, L)
    H = ref.interaction_energy(n, phi, 0.5, G)
    assert abs(cnt["energy"] - (H - c.E * cnt["P"])) <= 1e-9 * max(1.0, abs(H))
    # each logged pair moved two electrons to empty sites by disk vectors
    dxs, dys, _, _ = c.vectors()
    disk = set(zip(dxs.tolist(), dys.tolist()))
    for e in log[pair][:200]:
        assert (int(e["dx2"]), int(e["dy2"])) in disk
        assert len({int(e["i"]), int(e["j"]), int(e["k"]), int(e["l"])}) == 4


def test_zero_pair_fraction_is_the_single_hop_chain():
    a = oracle.Chain(16, 16, r_max=4, T=0.05, E=0.01, seed=7)
    b = oracle.Chain(16, 16, r_max=4, T=0.05, E=0.01, seed=7)
    b.set_pair(0.0, 3)
    assert b.pair_threshold == 0 and b.Gamma == a.Gamma
    _, la = a.run(1500, 256, log=True)
    _, lb = b.run(1500, 256, log=True)
    for f in ("i", "j", "q", "p", "round", "dx", "dy", "dE"):
        np.testing.assert_array_equal(la[f], lb[f])
    assert np.all(lb["k"] == 0xFFFFFFFF)
    np.testing.assert_array_equal(a.state()[1], b.state()[1])


def test_gamma_counts_the_pair_attempts():
    c = oracle.Chain(16, 16, r_max=4, T=0.05, seed=7, pair_frac=0.25, pair_rmax=3)
    Tp = c.pair_threshold
    assert Tp == 1 << 30
    assert c.Gamma == 256 * c.Z / (1.0 - Tp * 2.0 ** -32)
    with pytest.raises(ValueError):
        c.set_pair(1.0, 3)
    with pytest.raises(ValueError):
        c.set_pair(0.1, 8)          # 2R must stay below L
    with pytest.raises(ValueError):
        oracle.Chain(8, 1, r_max=2, pair_frac=0.1, pair_rmax=2)      # a ring has no pairs



# ---------------------------------------------------------------------------
# the cubic lattice: the offset's z is the fourth word of the pair block
# ---------------------------------------------------------------------------

def _pair_moves3(c, n, R):
    """Every 3D pair proposal with its probability given a pair label (offset
    uniform on the cube [-R, R]^3, kept with both offsets inside the ball):
    yields (prob, i, j, k, l, dx1, dx2)."""
    L, N = c.Lx, c.N
    dxs, dys, Wi, _ = c.vectors()
    dzs = c.vectors_z()
    pd = Wi.astype(np.float64) / 2.0 ** 32
    W = 2 * R + 1

    def site(x, y, z):
        return ((z % L) * L + (y % L)) * L + (x % L)
    for i in np.nonzero(n)[0]:
        xi, yi, zi = i % L, (i // L) % L, i // (L * L)
        for v1 in range(len(dxs)):
            j = site(xi + dxs[v1], yi + dys[v1], zi + dzs[v1])
            if n[j]:
                continue
            for ex, ey, ez in itertools.product(range(-R, R + 1), repeat=3):
                if not 0 < ex * ex + ey * ey + ez * ez <= R * R:
                    continue
                k = site(xi + ex, yi + ey, zi + ez)
                if not n[k]:
                    continue
                xk, yk, zk = k % L, (k // L) % L, k // (L * L)
                for v2 in range(len(dxs)):
                    l = site(xk + dxs[v2], yk + dys[v2], zk + dzs[v2])
                    if n[l]:
                        continue
                    f = (ex + dxs[v2] - dxs[v1], ey + dys[v2] - dys[v1], ez + dzs[v2] - dzs[v1])
                    f2 = f[0] ** 2 + f[1] ** 2 + f[2] ** 2
                    if not 0 < f2 <= R * R:
                        continue
                    yield ((1.0 / N) * pd[v1] * pd[v2] / W ** 3,
                           int(i), int(j), int(k), int(l), int(dxs[v1]), int(dxs[v2]))


def _kernel_row3(c, n, R, p2q, index):
    L, N = c.Lx, c.N
    dxs, dys, Wi, _ = c.vectors()
    dzs = c.vectors_z()
    pd = Wi.astype(np.float64) / 2.0 ** 32
    row = {}
    c.set_state(n)
    for i in np.nonzero(n)[0]:
        xi, yi, zi = i % L, (i // L) % L, i // (L * L)
        for v in range(len(dxs)):
            j = (((zi + dzs[v]) % L) * L + (yi + dys[v]) % L) * L + (xi + dxs[v]) % L
            if n[j]:
                continue
            acc = min(1.0, math.exp(-c.delta_e(i, j, int(dxs[v])) / c.T))
            n2 = n.copy()
            n2[i], n2[j] = 0, 1
            b = index[n2.tobytes()] if index is not None else n2.tobytes()
            row[b] = row.get(b, 0.0) + (1.0 - p2q) * (1.0 / N) * pd[v] * acc
    for prob, i, j, k, l, dx1, dx2 in _pair_moves3(c, n, R):
        acc = min(1.0, math.exp(-c.delta_e_pair(i, j, k, l, dx1, dx2) / c.T))
        n2 = n.copy()
        n2[i], n2[j], n2[k], n2[l] = 0, 1, 0, 1
        b = index[n2.tobytes()] if index is not None else n2.tobytes()
        row[b] = row.get(b, 0.0) + p2q * prob * acc
    return row


@pytest.mark.parametrize("E", [0.0, 0.05])
def test_pair_delta_e_on_the_cube(E):
    L = 6
    N = L ** 3
    c = oracle.Chain(L, dim=3, r_max=2, T=0.1, E=E, seed=2, pair_frac=0.3, pair_rmax=2)
    G = ref.coupling_matrix3(L, L, L)
    rng = np.random.default_rng(9)
    n = workloads.random_occupation(N, N // 2, seed=41)
    phi = workloads.random_phi(N, 1.0, seed=51)
    c.set_state(n, phi)
    H0 = ref.interaction_energy(n, phi, 0.5, G)
    moves = list(_pair_moves3(c, n, 2))
    for m in rng.choice(len(moves), 120, replace=False):
        _, i, j, k, l, dx1, dx2 = moves[m]
        n2 = n.copy()
        n2[i], n2[j], n2[k], n2[l] = 0, 1, 0, 1
        want = (ref.interaction_energy(n2, phi, 0.5, G) - H0) - E * (dx1 + dx2)
        assert abs(c.delta_e_pair(i, j, k, l, dx1, dx2) - want) <= 1e-12 * (1 + abs(H0) / N)


def test_pair_detailed_balance_on_the_cube():
    L, ne = 4, 2
    N = L ** 3
    c = oracle.Chain(L, dim=3, nu=ne / N, r_max=1, T=0.4, E=0.0, seed=6, pair_frac=0.4,
                     pair_rmax=1)
    _, _, phi = c.state()
    states = _states(N, ne)
    index = {s.tobytes(): a for a, s in enumerate(states)}
    G = ref.coupling_matrix3(L, L, L)
    H = ref.interaction_energy_batch(states, phi, ne / N, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    p2q = c.pair_threshold * 2.0 ** -32
    K = np.zeros((len(states), len(states)))
    for a, n in enumerate(states):
        for b, v in _kernel_row3(c, n, 1, p2q, index).items():
            K[a, b] += v
    K[np.diag_indices_from(K)] += 1.0 - K.sum(axis=1)
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    four = sum(1 for a, n in enumerate(states) for b in np.nonzero(K[a])[0]
               if np.abs(states[b].astype(int) - n).sum() == 4)
    assert four > 100          # pair moves are part of the kernel


def test_oracle_labels_follow_the_kernel_row_on_the_cube():
    # 16 electrons filling the 2 x 2 x 4 block x, y < 2 of a 4^3 torus: many
    # neighbouring pairs, including pairs along z (their offsets need ez)
    L = 4
    N = L ** 3
    c = oracle.Chain(L, dim=3, nu=16 / N, r_max=1, T=1.0, E=0.0, seed=4, pair_frac=0.9,
                     pair_rmax=1)
    n = np.zeros(N, np.uint8)
    for z in range(L):
        for y in range(2):
            for x in range(2):
                n[(z * L + y) * L + x] = 1
    c.set_state(n)
    row = _kernel_row3(c, n, 1, c.pair_threshold * 2.0 ** -32, None)
    n_labels = 400_000
    counts = {}
    for t in range(n_labels):
        lab = c.eval_label(t // 64, t % 64)
        if lab.accepted:
            n2 = n.copy()
            n2[lab.i], n2[lab.j] = 0, 1
            if lab.pair:
                n2[lab.k], n2[lab.l] = 0, 1
            b = n2.tobytes()
            counts[b] = counts.get(b, 0) + 1
    assert set(counts) <= set(row)
    is_pair = {b: int(np.abs(np.frombuffer(b, np.uint8).astype(int) - n).sum() == 4)
               for b in row}
    # all pair moves together: a binomial count
    p_pair = sum(pb for b, pb in row.items() if is_pair[b])
    got = sum(v for b, v in counts.items() if is_pair[b])
    assert abs(got - p_pair * n_labels) < 5 * math.sqrt(n_labels * p_pair), (got, p_pair)
    assert got > 200
    # every target with at least 5 expected hits
    chi2, dof, pair_bins = 0.0, 0, 0
    for b, pb in row.items():
        e = pb * n_labels
        if e >= 5:
            chi2 += (counts.get(b, 0) - e) ** 2 / e
            dof += 1
            pair_bins += is_pair[b]
    assert dof >= 10 and pair_bins >= 20, (dof, pair_bins)
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_pair_run_on_the_cube_keeps_eps_energy_and_dipole():
    L = 8
    c = oracle.Chain(L, dim=3, r_max=2, T=0.5, E=0.02, seed=3, pair_frac=0.6, pair_rmax=2)
    P0 = c.counters()["P"]
    rc, log = c.run(3000, 128, log=True)
    assert rc == oracle.ORC_OK
    assert (log["k"] != 0xFFFFFFFF).sum() > 10
    n, eps, phi = c.state()
    assert np.abs(eps - c.eps_scratch()).max() <= 1e-11
    cnt = c.counters()
    assert cnt["P"] - P0 == int(log["dx"].sum() + log["dx2"].sum())
    G = ref.coupling_matrix3(L, L, L)
    H = ref.interaction_energy(n, phi, 0.5, G)
    assert abs(cnt["energy"] - (H - c.E * cnt["P"])) <= 1e-9 * max(1.0, abs(H))
