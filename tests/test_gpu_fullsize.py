"""Parity at full size, in the launch configuration bench.py times: 304
replicas of L=128 (N=16384), T=0.01, W=2, r_max=8, E=0.005, binary32 eps with
the split-BF16 tensor-core refresh every 1024 hops, 512 threads per CTA, two
CTAs per SM, M=4096 (the L=128 workload of the mixed PR algorithm, section
"Hopping conduction in the Coulomb glass", batched).

Checked on every replica (properties that hold at any size): each logged hop
moves an electron from an occupied site to an empty one by a vector of the
hop disk, j = i + (dx, dy) on the torus, the replayed occupation equals the
device's, and the dipole and attempt counters are the sums over the log
(attempts += (p-1)M + q).  Checked on sampled replicas against the oracle:
every logged label's proposal (site, vector, destination) equals the
oracle's for the same (round, label), bit for bit; the binary64 serial chain
executes the same hops, or, where the two first differ, the label that
decides it sits at the Metropolis threshold within the binary32 eps error;
after the refresh eps is within 1e-4 of its definition.  The binary64 form
in the same batch shape is bit-exact on the sampled replicas.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_5026_gb300 import workloads

pytestmark = pytest.mark.gpu

R, L, M, HOPS, THREADS = 304, 128, 4096, 1024, 512
SAMPLED = (0, 151, 303)


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def _reps():
    return [r.as_dict() for r in workloads.l128_batch(R).replicas]


def _oracle_for(p):
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=p["seed"], replica=p.get("replica", 0))


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


@pytest.fixture(scope="module")
def fp32_run(B):
    reps = _reps()
    s = B.System(reps, precision=B.CG_FP32, refresh_every=HOPS,
                 refresh_kind=B.CG_REFRESH_BF16X2, block_threads=THREADS)
    try:
        start = [s.state(k) for k in range(R)]
        rc, log = s.run_logged(HOPS, M)
        assert rc == B.CG_OK
        end = [s.state(k) for k in range(R)]
        obs = [s.observables(k) for k in range(R)]
        shapes = [B.cg_group_shape(s.h, g) for g in range(B.cg_num_groups(s.h))]
    finally:
        s.close()
    return reps, start, log, end, obs, shapes


def test_launch_shape_is_the_bench_shape(fp32_run):
    *_, shapes = fp32_run
    assert shapes == [{"L": L, "threads": THREADS, "M": 4096, "cluster": 1}]


def test_every_replica_log_replays_to_its_state(fp32_run):
    reps, start, log, end, obs, _ = fp32_run
    ch = _oracle_for(reps[0])
    dx_v, dy_v, _, _ = ch.vectors()
    disk = set(zip(dx_v.tolist(), dy_v.tolist()))
    for k in range(R):
        n = start[k][0].astype(np.int8).copy()
        lg = log[k]
        i, j = lg["i"].astype(np.int64), lg["j"].astype(np.int64)
        dx, dy = lg["dx"].astype(np.int64), lg["dy"].astype(np.int64)
        assert np.all(((i % L) + dx) % L == j % L) and np.all(((i // L) + dy) % L == j // L)
        assert all((a, b) in disk for a, b in zip(dx.tolist(), dy.tolist()))
        for h in range(HOPS):
            assert n[i[h]] == 1 and n[j[h]] == 0, (k, h)
            n[i[h]] = 0
            n[j[h]] = 1
        np.testing.assert_array_equal(n, end[k][0])
        c0, c1 = start[k][3], end[k][3]
        assert c1["P"] - c0["P"] == int(dx.sum())
        m = (lg["p"].astype(np.int64) - 1) * M + lg["q"].astype(np.int64)
        assert c1["attempts"] - c0["attempts"] == int(m.sum())
        assert c1["hops"] - c0["hops"] == HOPS
        assert obs[k]["max_eps_err_last_refresh"] <= 1e-4


@pytest.mark.parametrize("k", SAMPLED)
def test_sampled_proposals_equal_the_oracle(fp32_run, k):
    reps, start, log, *_ = fp32_run
    ch = _oracle_for(reps[k])
    for h in range(0, HOPS, 7):
        e = log[k][h]
        lab = ch.eval_label(int(e["round"]), int(e["q"]) - 1)
        assert (lab.i, lab.j, lab.dx, lab.dy) == (e["i"], e["j"], e["dx"], e["dy"]), (k, h)


@pytest.mark.parametrize("k", SAMPLED)
def test_sampled_chain_follows_binary64_up_to_threshold_decisions(fp32_run, k):
    reps, start, log, end, obs, _ = fp32_run
    p = reps[k]
    ch = _oracle_for(p)
    _, olog = ch.run(HOPS, M, log=True)
    g = log[k]
    same = (g["round"] == olog["round"]) & (g["q"] == olog["q"])
    if same.all():
        # the whole trajectory agrees: the binary32 state matches the oracle
        n, eps, _, cnt = end[k]
        on, oeps, _ = ch.state()
        np.testing.assert_array_equal(n, on)
        assert np.max(np.abs(eps - oeps)) <= 1e-4
        return
    h = int(np.nonzero(~same)[0][0])
    # the state before hop h is common; the earlier of the two decisive labels
    # is accepted on one side and rejected on the other: it must sit at the
    # threshold, |ln u + dH/T| within what a binary32 eps error of 1e-4 on
    # both sites can move
    ref = _oracle_for(p)
    ref.run(h, M)
    a = (int(g[h]["round"]), int(g[h]["q"]))
    b = (int(olog[h]["round"]), int(olog[h]["q"]))
    rnd, q = min(a, b)
    lab = ref.eval_label(rnd, q - 1)
    assert lab.theta
    margin = abs(math.log(lab.u) + lab.dE / p["T"])
    assert margin <= 4e-4 / p["T"], (k, h, margin)


@pytest.mark.parametrize("k", SAMPLED)
def test_eps_after_refresh_matches_its_definition(fp32_run, k):
    reps, start, log, end, *_ = fp32_run
    n, eps, phi, _ = end[k]
    ch = _oracle_for(reps[k])
    ch.set_state(n, phi)
    exact = ch.state()[1]
    assert np.max(np.abs(eps - exact)) <= 1e-4


def test_binary64_in_the_batch_shape_is_bit_exact_on_sampled_replicas(B):
    reps = _reps()
    hops = 512
    s = B.System(reps, precision=B.CG_FP64, block_threads=1024)
    try:
        rc = s.run(hops, M)
        assert rc == B.CG_OK
        for k in SAMPLED:
            ch = _oracle_for(reps[k])
            ch.run(hops, M)
            n, eps, phi, cnt = s.state(k)
            on, oeps, ophi = ch.state()
            np.testing.assert_array_equal(n, on)
            np.testing.assert_array_equal(_bits(eps), _bits(oeps))
            oc = ch.counters()
            for f in ("rounds", "hops", "attempts", "P"):
                assert cnt[f] == oc[f], (k, f)
    finally:
        s.close()
