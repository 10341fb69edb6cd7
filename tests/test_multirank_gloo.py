"""The multi-GPU path of bench.py on CPU: two gloo ranks.

Replicas are independent chains, so ranks run disjoint replica sets and only
the timing is combined: the job time is the slowest rank's, hops and attempts
are summed.  No GPU is used.
"""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    reps = bench.replicas_for(rank, 3)
    # rank r pretends to take (r + 1) s for 100 (r + 1) hops
    t, h, a = bench.combine_ranks(float(rank + 1), 100 * (rank + 1), 1000 * (rank + 1))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"seeds": [r["seed"] for r in reps], "replicas": [r["replica"] for r in reps],
                   "t": t, "h": h, "a": a}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_replicas_and_combine_timing(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert set(r0["seeds"]).isdisjoint(r1["seeds"])
    assert r0["seeds"] == [0, 1, 2] and r1["seeds"] == [3, 4, 5]
    assert r0["replicas"] == r0["seeds"]
    for r in (r0, r1):
        assert r["t"] == 2.0          # the slowest rank
        assert r["h"] == 300.0 and r["a"] == 3000.0


def test_single_process_combine_is_identity():
    import bench
    assert bench.combine_ranks(1.5, 7, 9) == (1.5, 7.0, 9.0)
