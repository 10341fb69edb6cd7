"""Pins of the oracle on the cubic lattice (the three-dimensional extension
the paper names in its conclusions): the hop ball against a brute-force
count and its order (dz outermost, then the square lattice's dy, dx), the
folded 1/r table against closed forms, eps and dH against independent
numpy evaluations of Eq. 1 with minimum-image distances on the 3D torus,
the incremental eps of a run against eps from scratch, and detailed balance
of the serial chain by exact enumeration of every state of two electrons on
a 4 x 4 x 4 torus.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads
from tests import physics_ref as ref


@pytest.mark.parametrize("r_max", [1, 2, 3, 5])
def test_hop_ball_count_and_order(r_max):
    L = 2 * r_max + 2
    c = oracle.Chain(L, dim=3, r_max=r_max)
    want = [(dx, dy, dz) for dz, dy, dx in itertools.product(range(-r_max, r_max + 1), repeat=3)
            if 0 < dx * dx + dy * dy + dz * dz <= r_max * r_max]
    assert c.V == len(want)
    dx, dy, Wi, w = c.vectors()
    dz = c.vectors_z()
    assert list(zip(dx.tolist(), dy.tolist(), dz.tolist())) == want
    # weights depend on |d| only: equal for every vector of a shell
    r2 = dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2 + dz.astype(np.int64) ** 2
    for q in np.unique(r2):
        assert len(set(Wi[r2 == q].tolist())) == 1


def test_cubic_table_closed_forms():
    L = 10
    c = oracle.Chain(L, dim=3, r_max=2)
    t = c.tinv_table()
    assert t.shape == (6, 6, 6)
    assert t[0, 0, 0] == 0.0
    assert t[0, 0, 1] == 1.0 and t[1, 0, 0] == 1.0
    assert t[0, 1, 1] == 1.0 / math.sqrt(2.0)
    assert t[1, 1, 1] == 1.0 / math.sqrt(3.0)
    assert t[1, 1, 2] == 1.0 / math.sqrt(6.0)
    # minimum image along every axis
    for d in range(L):
        f = min(d, L - d)
        assert c.tinv(d, 0, 0) == c.tinv(f, 0, 0) == c.tinv(0, 0, d) == c.tinv(0, d, 0)
    assert c.tinv(L - 1, L - 1, L - 1) == 1.0 / math.sqrt(3.0)


@pytest.mark.parametrize("L,nu", [(4, 0.5), (6, 0.25)])
def test_eps_scratch_matches_dense_contraction_3d(L, nu):
    c = oracle.Chain(L, dim=3, nu=nu, r_max=1, seed=3)
    n, eps, phi = c.state()
    G = ref.coupling_matrix3(L, L, L)
    want = ref.site_energies(n, phi, nu, G)
    assert np.max(np.abs(eps - want)) <= 1e-12


@pytest.mark.parametrize("E", [0.0, 0.1])
def test_delta_e_equals_hamiltonian_difference_3d(E):
    L = 4
    N = L ** 3
    c = oracle.Chain(L, dim=3, r_max=1, T=0.1, E=E, seed=2)
    G = ref.coupling_matrix3(L, L, L)
    dxs, dys, _, _ = c.vectors()
    dzs = c.vectors_z()
    rng = np.random.default_rng(5)
    for trial in range(3):
        n = workloads.random_occupation(N, N // 2, seed=10 + trial)
        phi = workloads.random_phi(N, 1.0, seed=20 + trial)
        c.set_state(n, phi)
        H0 = ref.interaction_energy(n, phi, 0.5, G)
        occ = np.where(n == 1)[0]
        for _ in range(60):
            i = int(rng.choice(occ))
            k = int(rng.integers(len(dxs)))
            x, y, z = i % L, (i // L) % L, i // (L * L)
            j = (((z + dzs[k]) % L) * L + (y + dys[k]) % L) * L + (x + dxs[k]) % L
            if n[j] == 1:
                continue
            n2 = n.copy()
            n2[i], n2[j] = 0, 1
            want = (ref.interaction_energy(n2, phi, 0.5, G) - H0) - E * dxs[k]
            assert abs(c.delta_e(i, j, int(dxs[k])) - want) <= 1e-12 * (1 + abs(H0) / N)


def test_incremental_eps_equals_scratch_3d():
    c = oracle.Chain(8, dim=3, r_max=2, T=0.1, E=0.02, seed=7)
    c.run(3000, 256)
    n, eps, phi = c.state()
    scratch = c.eps_scratch()
    assert np.max(np.abs(eps - scratch)) <= 1e-11
    # the running energy follows Eq. 1 evaluated from scratch (the field
    # term uses the unwrapped dipole)
    G = ref.coupling_matrix3(8, 8, 8)
    cnt = c.counters()
    H = ref.interaction_energy(n, phi, 0.5, G)
    H0_field = c.E * (cnt["P"])
    assert abs(cnt["energy"] - (H - H0_field)) <= 1e-9 * max(1.0, abs(H))


def test_detailed_balance_two_electrons_on_a_cube():
    L, k = 4, 2
    N = L ** 3
    c = oracle.Chain(L, dim=3, nu=k / N, r_max=1, T=0.3, E=0.0, seed=6)
    _, _, phi = c.state()
    states = []
    for occ in itertools.combinations(range(N), k):
        n = np.zeros(N, np.uint8)
        n[list(occ)] = 1
        states.append(n)
    states = np.array(states)
    G = ref.coupling_matrix3(L, L, L)
    H = ref.interaction_energy_batch(states, phi, k / N, G)
    pi = np.exp(-(H - H.min()) / c.T)
    pi /= pi.sum()
    dxs, dys, Wi, _ = c.vectors()
    dzs = c.vectors_z()
    pd = Wi.astype(np.float64) / 2.0 ** 32
    index = {s.tobytes(): a for a, s in enumerate(states)}
    K = np.zeros((len(states), len(states)))
    for a, n in enumerate(states):
        c.set_state(n, phi)
        for i in np.nonzero(n)[0]:
            x, y, z = i % L, (i // L) % L, i // (L * L)
            for q in range(len(dxs)):
                j = (((z + dzs[q]) % L) * L + (y + dys[q]) % L) * L + (x + dxs[q]) % L
                if n[j]:
                    continue
                acc = min(1.0, math.exp(-c.delta_e(int(i), int(j), int(dxs[q])) / c.T))
                n2 = n.copy()
                n2[i], n2[j] = 0, 1
                K[a, index[n2.tobytes()]] += (1.0 / N) * pd[q] * acc
    K[np.diag_indices_from(K)] += 1.0 - K.sum(axis=1)
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()


@pytest.mark.parametrize("L", [4, 6])
def test_fft_reference_matches_dense_3d(L):
    # the FFT form of eps used by the GPU refresh tests equals the dense
    # contraction with the minimum-image coupling matrix
    N = L ** 3
    n = workloads.random_occupation(N, N // 2, seed=L)
    phi = workloads.random_phi(N, 1.0, seed=L + 1)
    dense = ref.site_energies(n, phi, 0.5, ref.coupling_matrix3(L, L, L))
    assert np.abs(ref.site_energies_fft3(n, phi, 0.5, L) - dense).max() <= 1e-12
