"""Writes tests/golden/oracle_*.json by running the CPU oracle only.

Usage: python tests/golden/make_oracle_golden.py
The stored values are regression pins of the oracle itself (its counters and
a digest of its state after a fixed run); they come from ``oracle/`` alone.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from numpy.lib.recfunctions import repack_fields  # noqa: E402


def summary(Lx, nu, W, xi, r_max, T, E, seed, M, hops):
    c = oracle.Chain(Lx, nu=nu, W=W, xi=xi, r_max=r_max, T=T, E=E, seed=seed)
    rc, log = c.run(hops, M, log=True)
    n, eps, phi = c.state()
    return {
        "params": dict(L=Lx, nu=nu, W=W, xi=xi, r_max=r_max, T=T, E=E, seed=seed,
                       M=M, hops=hops),
        "status": rc,
        "counters": c.counters(),
        "n_sha256": hashlib.sha256(n.tobytes()).hexdigest(),
        "eps_sha256": hashlib.sha256(eps.tobytes()).hexdigest(),
        # the single-hop fields of each log record, packed in this order
        "log_sha256": hashlib.sha256(repack_fields(
            log[["i", "j", "q", "p", "round", "dx", "dy", "dE"]]).tobytes()).hexdigest(),
        "first_hops": [[int(h["i"]), int(h["j"]), int(h["q"]), int(h["p"])]
                       for h in log[:8]],
    }


def main():
    out = summary(16, 0.5, 1.0, 1.0, 4, 0.05, 0.0, 0, 256, 10_000)
    out["cite"] = ("L=16 half-filled 2D lattice Coulomb glass (section 'Results "
                   "for the lattice model in two dimensions'), mixed algorithm "
                   "of the section 'Hopping conduction in the Coulomb glass'")
    with open(os.path.join(HERE, "oracle_l16_1e4.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
