"""Oracle chains for a process pool (started with the spawn method): each
worker builds its chain from plain parameters and returns the final state."""


def run_chain(args):
    p, hops, M = args
    import oracle
    ch = oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"], T=p["T"],
                      E=p["E"], seed=p["seed"], replica=p.get("replica", 0))
    rc, _ = ch.run(hops, M)
    n, eps, _ = ch.state()
    return rc, n, eps, ch.counters()
