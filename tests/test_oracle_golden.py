"""Stored pins: the paper's Fig. 1 worked example and a regression digest of
the oracle (written by tests/golden/make_oracle_golden.py from oracle/ only)."""
import hashlib
import json
import os

import numpy as np
from numpy.lib.recfunctions import repack_fields

import oracle

LOG_FIELDS = ("i", "j", "q", "p", "round", "dx", "dy", "dE")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_fig1_attempt_count():
    g = json.load(open(os.path.join(GOLDEN, "fig1_example.json")))
    # the reading (p-1) M + q reproduces the caption's serial iteration count
    assert (g["p"] - 1) * g["M"] + g["q"] == g["m"]
    # a chain in which the first accept sits at round 2, label 5 of M = 12:
    # constant-acceptance mode with the oracle's own bookkeeping
    c = oracle.Chain(16, r_max=4, seed=0)
    c.set_toy(0.5)
    found = False
    for seed in range(2000):
        c = oracle.Chain(16, r_max=4, seed=seed)
        c.set_toy(0.08)
        rc, log = c.run(1, g["M"], log=True)
        if log[0]["p"] == g["p"] and log[0]["q"] == g["q"]:
            assert c.counters()["attempts"] == g["m"]
            found = True
            break
    assert found


def test_oracle_regression_digest():
    g = json.load(open(os.path.join(GOLDEN, "oracle_l16_1e4.json")))
    p = g["params"]
    c = oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                     T=p["T"], E=p["E"], seed=p["seed"])
    rc, log = c.run(p["hops"], p["M"], log=True)
    assert rc == g["status"]
    cnt = c.counters()
    for k, v in g["counters"].items():
        assert cnt[k] == v, k
    n, eps, _ = c.state()
    assert hashlib.sha256(n.tobytes()).hexdigest() == g["n_sha256"]
    assert hashlib.sha256(eps.tobytes()).hexdigest() == g["eps_sha256"]
    # the digest covers the single-hop fields of the log record
    base = repack_fields(log[list(LOG_FIELDS)])
    assert hashlib.sha256(base.tobytes()).hexdigest() == g["log_sha256"]
