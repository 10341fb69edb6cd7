"""Pins of the oracle's energies and chain against Eq. 1 and exact results.

* eps from scratch equals phi + G (n - nu) with G built by numpy from
  minimum-image ``hypot`` distances (definition below Eq. 2).
* dH of every hop equals H(beta) - H(alpha) - E dx from Eq. 1.
* the incremental eps update (step 3b) stays equal to a from-scratch eps.
* the running energy equals Eq. 1 re-evaluated on the current configuration.
"""
import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads
from tests import physics_ref as ref


@pytest.mark.parametrize("Lx,Ly,nu", [(8, 8, 0.5), (10, 6, 0.5), (8, 1, 0.5),
                                      (12, 12, 0.25)])
def test_eps_scratch_matches_dense_contraction(Lx, Ly, nu):
    c = oracle.Chain(Lx, Ly, nu=nu, W=1.3, r_max=1 if Ly == 1 else 2, T=0.1, seed=3)
    n, eps, phi = c.state()
    assert int(n.sum()) == round(nu * Lx * Ly)
    G = ref.coupling_matrix(Lx, Ly)
    np.testing.assert_allclose(eps, ref.site_energies(n, phi, nu, G), rtol=0,
                               atol=1e-12)
    # setting an arbitrary state rebuilds eps the same way
    n2 = workloads.random_occupation(Lx * Ly, int(n.sum()), seed=11)
    phi2 = workloads.random_phi(Lx * Ly, 2.0, seed=12)
    c.set_state(n2, phi2)
    _, eps2, _ = c.state()
    np.testing.assert_allclose(eps2, ref.site_energies(n2, phi2, nu, G), rtol=0,
                               atol=1e-12)


def test_disorder_and_initial_occupation_distribution():
    c = oracle.Chain(64, nu=0.5, W=2.0, r_max=4, seed=5)
    n, _, phi = c.state()
    assert n.sum() == 2048
    assert phi.min() >= -1.0 and phi.max() <= 1.0
    # uniform on [-W/2, W/2]: Kolmogorov-Smirnov distance small
    xs = np.sort(phi)
    F = (xs + 1.0) / 2.0
    ks = np.max(np.abs(F - (np.arange(1, len(xs) + 1) / len(xs))))
    assert ks < 1.95 / np.sqrt(len(xs))       # alpha ~ 0.001
    # occupied sites spread evenly over the lattice halves
    half = n.reshape(64, 64)
    assert abs(int(half[:32].sum()) - 1024) < 120
    # different replica -> different disorder
    c2 = oracle.Chain(64, nu=0.5, W=2.0, r_max=4, seed=5, replica=1)
    assert not np.array_equal(c2.state()[2], phi)


@pytest.mark.parametrize("E", [0.0, 0.07, -0.2])
def test_delta_e_equals_hamiltonian_difference(E):
    Lx = Ly = 8
    c = oracle.Chain(Lx, Ly, nu=0.5, W=1.0, r_max=3, T=0.1, E=E, seed=1)
    G = ref.coupling_matrix(Lx, Ly)
    rng = np.random.default_rng(0)
    for trial in range(4):
        n = workloads.random_occupation(64, 32, seed=100 + trial)
        phi = workloads.random_phi(64, 1.0, seed=200 + trial)
        c.set_state(n, phi)
        H0 = ref.interaction_energy(n, phi, 0.5, G)
        dxs, dys, _, _ = c.vectors()
        occ = np.where(n == 1)[0]
        for _ in range(60):
            i = int(rng.choice(occ))
            k = int(rng.integers(len(dxs)))
            xi, yi = i % Lx, i // Lx
            j = ((yi + dys[k]) % Ly) * Lx + (xi + dxs[k]) % Lx
            if n[j] == 1:
                continue
            n2 = n.copy()
            n2[i], n2[j] = 0, 1
            H1 = ref.interaction_energy(n2, phi, 0.5, G)
            want = (H1 - H0) - E * dxs[k]
            got = c.delta_e(i, j, int(dxs[k]))
            assert abs(got - want) <= 1e-12 * (1 + abs(H0) / 64), (got, want)


@pytest.mark.parametrize("L,r_max,T,E,hops", [(16, 4, 0.05, 0.0, 10_000),
                                              (16, 4, 0.3, 0.05, 10_000),
                                              (12, 3, 0.1, 0.01, 5_000)])
def test_incremental_eps_equals_scratch(L, r_max, T, E, hops):
    c = oracle.Chain(L, nu=0.5, W=1.0, r_max=r_max, T=T, E=E, seed=7)
    rc, log = c.run(hops, 64, log=True)
    assert rc == oracle.ORC_OK
    n, eps, phi = c.state()
    np.testing.assert_allclose(eps, c.eps_scratch(), rtol=0, atol=1e-12)
    G = ref.coupling_matrix(L, L)
    np.testing.assert_allclose(eps, ref.site_energies(n, phi, 0.5, G), rtol=0,
                               atol=1e-12)
    cnt = c.counters()
    # running energy: Eq. 1 on the torus minus the field times the unwrapped dipole
    H_int = ref.interaction_energy(n, phi, 0.5, G)
    assert abs(cnt["energy"] - (H_int - E * cnt["P"])) <= 1e-9
    # the dipole is the sum of the executed hops' dx
    n0 = oracle.Chain(L, nu=0.5, W=1.0, r_max=r_max, T=T, E=E, seed=7).state()[0]
    P0 = int((np.arange(L * L) % L)[n0 == 1].sum())
    assert cnt["P"] == P0 + int(log["dx"].sum())
    # attempt accounting: (p-1) M + q per hop
    assert cnt["attempts"] == int(((log["p"].astype(np.int64) - 1) * 64 + log["q"]).sum())
    assert cnt["hops"] == hops
    # every executed hop moved an electron to an empty site
    nn = n0.copy()
    for h in log:
        assert nn[h["i"]] == 1 and nn[h["j"]] == 0
        nn[h["i"]], nn[h["j"]] = 0, 1
    np.testing.assert_array_equal(nn, n)


def test_field_drives_dipole_along_field():
    # linear response: P grows along the sign of E (section on conductivity)
    drift = {}
    for E in (0.05, -0.05):
        c = oracle.Chain(16, nu=0.5, W=1.0, r_max=4, T=0.2, E=E, seed=2)
        P0 = c.counters()["P"]
        c.run(20_000, 32)
        drift[E] = c.counters()["P"] - P0
    assert drift[0.05] > 200 and drift[-0.05] < -200


@pytest.mark.parametrize("L", [6, 10, 16])
def test_fft_site_energies_equal_dense_contraction(L):
    # the torus convolution used for large-L checks equals the dense G (n - nu)
    n = workloads.random_occupation(L * L, L * L // 2, seed=L)
    phi = workloads.random_phi(L * L, 1.0, seed=L + 1)
    a = ref.site_energies(n, phi, 0.5, ref.coupling_matrix(L, L))
    b = ref.site_energies_fft(n, phi, 0.5, L)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
