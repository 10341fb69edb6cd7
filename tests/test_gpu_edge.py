"""Edge cases of the chain on the GPU, bit-exact against the serial oracle in
binary64 (the mixed PR algorithm, section "Hopping conduction in the
Coulomb glass"): an empty run, the smallest lattice and hop disk, a single
electron and a single hole (theta almost never holds), a temperature at
which nearly every proposal with theta is accepted, a field strong enough
to dominate dH, a hop disk reaching just below L/2, fillings other than one
half, and lattice sides that are not powers of two; in binary32, a lattice
whose N is not a multiple of the tensor-core tile (binary64 refresh).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _oracle_for(p):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0))


def _same_chain(B, p, hops, M, **kw):
    s = B.System([p], precision=B.CG_FP64, **kw)
    try:
        rc, log = s.run_logged(hops, M)
        assert rc == B.CG_OK
        ch = _oracle_for(p)
        _, olog = ch.run(hops, M, log=True)
        for f in ("i", "j", "q", "p", "round", "dx", "dy"):
            np.testing.assert_array_equal(log[0][f], olog[f], err_msg=f)
        np.testing.assert_array_equal(_bits(log[0]["dE"]), _bits(olog["dE"]))
        n, eps, _, cnt = s.state(0)
        on, oeps, _ = ch.state()
        np.testing.assert_array_equal(n, on)
        np.testing.assert_array_equal(_bits(eps), _bits(oeps))
        oc = ch.counters()
        for f in ("rounds", "hops", "attempts", "P"):
            assert cnt[f] == oc[f], f
        return cnt
    finally:
        s.close()


BASE = dict(nu=0.5, W=1.0, xi=1.0, T=0.05, E=0.01, seed=3)


def test_zero_hops_leaves_the_state_unchanged(B):
    p = dict(BASE, L=16, r_max=4)
    s = B.System([p], precision=B.CG_FP64)
    try:
        before = s.state(0)
        assert s.run(0, 1024) == B.CG_OK
        after = s.state(0)
        np.testing.assert_array_equal(before[0], after[0])
        np.testing.assert_array_equal(_bits(before[1]), _bits(after[1]))
        assert before[3] == after[3]
    finally:
        s.close()


@pytest.mark.parametrize("case", [
    dict(L=4, r_max=1),                       # smallest lattice, 4 hop vectors
    dict(L=6, r_max=2),                       # non-power-of-two, tiny
    dict(L=10, r_max=4),
    dict(L=18, r_max=8),                      # hop disk just below L/2
    dict(L=16, r_max=7, xi=2.5),              # long tunnelling length
], ids=lambda c: f"L{c['L']}_r{c['r_max']}")
def test_small_and_odd_lattices(B, case):
    p = dict(BASE, **case)
    _same_chain(B, p, 1500, 128)


@pytest.mark.parametrize("nu_n", [1, -1], ids=["one_electron", "one_hole"])
def test_single_electron_and_single_hole(B, nu_n):
    L = 8
    N = L * L
    nu = (1 if nu_n == 1 else N - 1) / N
    p = dict(BASE, L=L, r_max=3, nu=nu, T=0.2)
    cnt = _same_chain(B, p, 300, 64)
    # theta holds for about one proposal in N: hops take many labels
    assert cnt["attempts"] > 10 * cnt["hops"]


def test_quarter_filling(B):
    p = dict(BASE, L=16, r_max=4, nu=0.25)
    _same_chain(B, p, 1200, 200)


def test_high_temperature_accepts_almost_every_theta(B):
    p = dict(BASE, L=16, r_max=4, T=1000.0)
    cnt = _same_chain(B, p, 2000, 32)
    # theta holds for about nu (1 - nu) = 1/4 of the proposals
    assert cnt["attempts"] < 6 * cnt["hops"]


def test_strong_field_dominates(B):
    p = dict(BASE, L=16, r_max=4, E=5.0, T=0.1)
    cnt = _same_chain(B, p, 800, 256)
    assert cnt["P"] > 0      # hops run along the field


def test_binary32_lattice_without_tensor_core_tiles(B):
    # N = 18^2 = 324 is not a multiple of 128: the refresh runs in binary64
    reps = [dict(BASE, L=18, r_max=6, T=0.02, seed=s, replica=s) for s in range(10)]
    s = B.System(reps, precision=B.CG_FP32, refresh_every=256)
    try:
        s.run(2000, 512)
        for k in range(10):
            o = s.observables(k)
            assert o["refreshes"] >= 7 and 0 < o["max_eps_err_last_refresh"] <= 1e-4
            n, eps, phi, _ = s.state(k)
            ch = _oracle_for(reps[k])
            ch.set_state(n, phi)
            assert np.max(np.abs(eps - ch.state()[1])) <= 1e-4
    finally:
        s.close()


def test_lattice_beyond_any_cluster_is_refused(B):
    # L = 512 in binary32: eps is 1 MiB and the folded table alone 264 KB,
    # more than one CTA's shared memory; the handle is refused on the host
    p = dict(BASE, L=512, r_max=6)
    with pytest.raises(B.CgError) as ei:
        B.System([p], precision=B.CG_FP32)
    assert ei.value.code == B.CG_EINVAL and "shared memory" in str(ei.value)
