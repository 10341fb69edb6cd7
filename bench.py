#!/usr/bin/env python
"""Benchmark of the parallel-rejection KMC hot path on one node.

Metric: accepted hops/s (and serial-equivalent attempts/s) of the L=128
(N=16384), T=0.01 lattice Coulomb glass (nu=1/2, phi ~ U[-1,1], xi=1,
r_max=8, E=0.005), binary32 eps with a binary64 refresh every 1024 hops, R
disorder replicas per GPU in one persistent launch; the plain binary64 form of
the same workload (one replica) is measured beside it.

A step: every replica executes 1024 hops (one refresh period: proposals,
acceptance, lowest accepting label, commit, eps update) and then the eps
refresh.  Inputs (tables, disorder, initial random configuration) are built
once; the timed region starts with the state resident in device memory.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

For N > 1 launch with torch.distributed.run; ranks run disjoint replica sets
(replicas only, no collective on the data path).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "accepted hops/s & equiv. attempts/s at L=128 T=0.01, FP32-batched vs FP64 form"
WORKLOAD = dict(L=128, nu=0.5, W=2.0, xi=1.0, r_max=8, T=0.01, E=0.005)
HOPS_PER_STEP = 1024          # one refresh period
L2_FLUSH_BYTES = 256 << 20    # > 129 MB L2

# DRAM bytes (read + write) of one launch of the persistent kernel in this
# workload (304 replicas x 1024 hops), from an ncu capture of the relaxed
# L=128 batch; valid only while the kernel sources hash to the captured
# version and the launch takes the captured kernel instance (CTA size and
# CTAs per replica).  M changes which labels are drawn, not the bytes (the
# state is loaded and stored once per launch): captures at M = 4096 and
# 16384 gave 20.748 and 20.742 MB.
TRAFFIC_CAPTURE = {"sources_sha256_16": "651cca43504ee42b", "bytes_per_launch": 20.752e6,
                   "replicas": 304, "hops_per_replica": 1024, "M": 16384, "threads": 512,
                   "cluster": 1}


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("cg_pr_kernel.cu", "cg_pr_persistent.cuh", "cg_pr_common.cuh", "cg_device.cuh"):
        with open(os.path.join(ROOT, "paper_1407_5026_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--replicas", type=int, default=0, help="per GPU; 0 = 2 per SM")
    ap.add_argument("--M", type=int, default=4096,
                    help="labels per round while relaxing (and in the timed steps with --no-tune)")
    ap.add_argument("--no-tune", action="store_true",
                    help="time with --M and the default launch shape instead of the autotuned one")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--fp64-hops", type=int, default=3000)
    ap.add_argument("--relax-steps", type=int, default=40,
                    help="untimed steps from the random start before warm-up")
    ap.add_argument("--obs-samples", type=int, default=64,
                    help="disorder samples of the binary32-vs-binary64 observable check (0: skip)")
    ap.add_argument("--obs-hops", type=int, default=32768)
    ap.add_argument("--no-other-configs", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-m-sweep", action="store_true")
    ap.add_argument("--config", default=None,
                    help="run only the named other configuration (e.g. cubic_L32_T0.05_R152) "
                         "and print its result as one JSON line")
    ap.add_argument("--sigma-hops", type=int, default=200_000,
                    help="hops per replica of the L=256 sigma(t) comparison (0 skips it)")
    ap.add_argument("--sigma-l64-hops", type=int, default=1_000_000,
                    help="hops per chain of the L=64 sigma(t) relaxation and its Eq. 4 "
                         "rescaling (3 temperatures x 8 disorder seeds; 0 skips it)")
    ap.add_argument("--clocks-dir", default=None,
                    help="folder for the raw nvidia-smi clock samples (default: the temp folder)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(total_s, hops, attempts, device=None):
    """Whole-job numbers over the ranks: the slowest rank's time, summed hops
    and attempts (replicas only: no collective touches the chains)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return total_s, float(hops), float(attempts)
    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    s = torch.tensor([float(hops), float(attempts)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t[0]), float(s[0]), float(s[1])


class _nvtx_range:
    """An NVTX range (no-op where torch has no NVTX)."""

    def __init__(self, name):
        import torch
        try:
            torch.cuda.nvtx.range_push(name)
            self.on = True
        except Exception:
            self.on = False

    def close(self):
        import torch
        if self.on:
            torch.cuda.nvtx.range_pop()


def default_replicas():
    """Replicas per GPU of the workload: two per SM (one per CTA, two CTAs
    resident per SM)."""
    try:
        import torch
        if torch.cuda.is_available():
            return 2 * torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        pass
    return 304


def workload_config(args, R):
    """The workload both arms name (the reference arm times a bounded sample
    of it on the host cores, described in its cpu_baseline)."""
    return {"workload": "L128_T0.01_fp32_batched", "L": 128, "T": 0.01,
            "replicas_per_gpu": R, "hops_per_replica_per_step": HOPS_PER_STEP,
            "M": (args.M if args.no_tune
                  else "autotuned from {1024, 4096, 16384, 65536} (relaxing with "
                       f"{args.M})"),
            "refresh": "every 1024 hops: eps from its definition by the convolution "
                       "theorem (binary32 radix-2 FFTs, two replicas per complex "
                       "transform, times DFT(1/r); phi added in binary64)",
            "l2": "256 MB buffer zeroed between steps (outside the timed events)",
            "state": f"chains relaxed {args.relax_steps * HOPS_PER_STEP} hops from "
                     f"their random start, then {args.warmup} warm-up steps"}


def replicas_for(rank, R):
    from paper_1407_5026_gb300.workloads import Replica
    base = rank * R
    return [Replica(seed=base + k, replica=base + k, **WORKLOAD).as_dict() for k in range(R)]


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device, folder=None):
        import tempfile
        self.device = device
        self.proc = None
        self.path = os.path.join(folder or tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# --------------------------------------------------------------------------

def _oracle_chain(seed):
    import oracle
    p = dict(WORKLOAD)
    return oracle.Chain(p["L"], nu=p["nu"], W=p["W"], xi=p["xi"], r_max=p["r_max"],
                        T=p["T"], E=p["E"], seed=seed, replica=seed)


def cpu_baseline(seconds, M, relax_hops):
    """The oracle as it stands, one chain on one core: relaxed untimed as many
    hops from its random start as the GPU arm's chains (so both are timed at
    the same chain age and acceptance), then timed for a bounded number of
    seconds."""
    ch = _oracle_chain(0)
    ch.run(relax_hops, M)
    c0 = ch.counters()
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        ch.run(16, M)
    dt = time.perf_counter() - t0
    c = ch.counters()
    hops, att = c["hops"] - c0["hops"], c["attempts"] - c0["attempts"]
    return {"value": hops / dt, "unit": "hops/s", "cores": 1, "kind": "oracle",
            "attempts_per_s": att / dt, "acceptance": hops / max(1, att),
            "sample": (f"replica seed 0 of the L=128 T=0.01 workload, hops "
                       f"{c0['hops']}..{c['hops']} (relaxed {relax_hops} hops from its "
                       f"random initial configuration, untimed), M={M}, {dt:.1f} s, binary64")}


_worker_chain = None


def _ref_init(seed, M, relax_hops):
    global _worker_chain
    _worker_chain = _oracle_chain(seed)
    _worker_chain.run(relax_hops, M)      # relaxed before any step is timed


def _ref_step(args):
    hops, M = args
    t0 = time.perf_counter()
    c0 = _worker_chain.counters()
    _worker_chain.run(hops, M)
    c1 = _worker_chain.counters()
    return c1["hops"] - c0["hops"], c1["attempts"] - c0["attempts"], time.perf_counter() - t0


def run_reference(args):
    """The oracle timed as the reference arm: one chain per host core."""
    import multiprocessing as mp
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    hops_per_chain = 256
    relax = args.relax_steps * HOPS_PER_STEP
    pools = [ctx.Pool(1, initializer=_ref_init, initargs=(s, args.M, relax))
             for s in range(cores)]
    try:
        def step():
            res = [p.apply_async(_ref_step, ((hops_per_chain, args.M),)) for p in pools]
            return [r.get() for r in res]
        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        hops = att = 0
        for _ in range(args.steps):
            for h, a, _dt in step():
                hops += h
                att += a
        dt = time.perf_counter() - t0
    finally:
        for p in pools:
            p.terminate()
    value = hops / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "hops/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "attempts_per_s": att / dt,
        "config": workload_config(args, args.replicas or default_replicas()),
        "acceptance": hops / max(1, att),
        "cpu_baseline": {"value": value, "unit": "hops/s", "cores": cores, "kind": "oracle",
                         "attempts_per_s": att / dt,
                         "sample": f"{cores} chains (seeds 0..{cores - 1}), each relaxed "
                                   f"{relax} hops from its random initial "
                                   f"configuration (untimed), then {hops_per_chain} hops per "
                                   f"chain per step"},
        "e2e": {"value": value, "unit": "hops/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1407_5026_gb300 import binding as B
    from paper_1407_5026_gb300 import build as libbuild

    ws, rank, local = dist_env()
    libbuild.build()
    B.load()
    # the tuned launch shape of the batch is cached, so the end-to-end batch
    # (same replicas) reuses it
    import tempfile
    os.environ.setdefault("CG_TUNE_CACHE", os.path.join(
        tempfile.gettempdir(), f"cg_tune_bench_{os.getpid()}.json"))
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    if args.config:
        # one of the other configurations alone (profiling runs)
        torch.cuda.set_device(local)
        print(json.dumps({"config": args.config,
                          "result": other_configs(args, B, local, only=args.config)}))
        return
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    R = args.replicas or 2 * sms
    reps = replicas_for(rank, R)
    N = WORKLOAD["L"] ** 2

    # peaks that bound the eps update (measured on this GPU)
    smem_peak = B.cg_microbench(0, local)          # bytes/s, 32-bit RMW
    dadd_peak = B.cg_microbench(1, local)          # adds/s
    philox_peak = B.cg_microbench(3, local)        # Philox blocks/s: one per evaluated label
    # seconds per barrier: one CTA of 1024 threads, clusters of 2, 4 and 8
    barrier_us = {c: B.cg_microbench(k, local) * 1e6 for c, k in ((1, 7), (2, 4), (4, 5), (8, 6))}

    sysm = B.System(reps, precision=B.CG_FP32, refresh_every=0, block_threads=args.threads,
                    device=local)
    st = sysm.stream
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")

    def one_step(ev, M):
        with torch.cuda.stream(st):
            if ev:
                ev[0].record(st)
            B.cg_run_async(sysm.h, HOPS_PER_STEP, M)
            if ev:
                ev[1].record(st)
            B.cg_refresh_async(sysm.h)
            if ev:
                ev[2].record(st)

    # relax every chain from its random start into the low-acceptance regime
    # (same steps as the timed ones, untimed)
    for _ in range(args.relax_steps):
        one_step(None, args.M)
        rc = B.cg_sync(sysm.h)
        assert rc == B.CG_OK, rc
    # the launch shape (M, CTA size, CTAs per replica) from the library's
    # autotuner on the relaxed batch (trials on a copy of the state; the
    # chains are left as they were); cg_run with M = 0 then uses it
    M_run = args.M
    if not args.no_tune:
        B.cg_autotune(sysm.h, HOPS_PER_STEP)
        M_run = 0
    shape = B.cg_group_shape(sysm.h, 0)
    for _ in range(args.warmup):
        one_step(None, M_run)
        rc = B.cg_sync(sysm.h)
        assert rc == B.CG_OK, rc
    obs0 = [B.cg_observables(sysm.h, k) for k in range(R)]

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local, args.clocks_dir)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    # an NVTX range around the timed steps lets a profiler select their
    # launches (ncu --nvtx --nvtx-include "timed_steps/")
    nvtx = _nvtx_range("timed_steps")
    for k in range(args.steps):
        one_step(events[k], M_run)
        with torch.cuda.stream(st):
            flush.zero_()                      # L2 flush between steps, outside the events
    nvtx.close()
    rc = B.cg_sync(sysm.h)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    assert rc == B.CG_OK, rc

    run_ms = [e[0].elapsed_time(e[1]) for e in events]
    ref_ms = [e[1].elapsed_time(e[2]) for e in events]
    step_ms = [a + b for a, b in zip(run_ms, ref_ms)]
    total_s = sum(step_ms) * 1e-3
    obs1 = [B.cg_observables(sysm.h, k) for k in range(R)]
    hops = sum(o1["hops"] - o0["hops"] for o0, o1 in zip(obs0, obs1))
    attempts = sum(o1["attempts"] - o0["attempts"] for o0, o1 in zip(obs0, obs1))
    evaluated = sum(o1["evaluated"] - o0["evaluated"] for o0, o1 in zip(obs0, obs1))
    cyc_upd = sum(o1["cycles_update"] - o0["cycles_update"] for o0, o1 in zip(obs0, obs1))
    cyc_rej = sum(o1["cycles_reject"] - o0["cycles_reject"] for o0, o1 in zip(obs0, obs1))
    max_err = max(o["max_eps_err_last_refresh"] for o in obs1)

    total_s_all, hops_all, att_all = combine_ranks(total_s, hops, attempts,
                                                   device=f"cuda:{local}")

    # roofline of the dominant kernel (the persistent PR kernel): algorithmic
    # bytes of the eps update per launch / mean launch time
    bytes_per_hop = N * (2 * 4 + 2 * 4)
    launch_s = statistics.mean(run_ms) * 1e-3
    achieved = R * HOPS_PER_STEP * bytes_per_hop / launch_s
    upd_s_per_cta = (cyc_upd / R) / (clk["sm_mhz"] * 1e6) if clk else None

    result = {
        "metric": METRIC, "value": hops_all / total_s_all, "unit": "hops/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "attempts_per_s": att_all / total_s_all,
        "acceptance": attempts and hops / attempts,
        "labels_evaluated_per_s": evaluated / total_s,
        "config": workload_config(args, R),
        "launch_shape": dict(shape, how=("cg_autotune on the relaxed batch" if not args.no_tune
                                         else "default launch shape, M from --M")),
        "roofline": {"bound": "smem", "achieved": achieved / 1e9, "peak": smem_peak / 1e9,
                     "unit": "GB/s", "frac": achieved / smem_peak,
                     "traffic": (TRAFFIC_CAPTURE["bytes_per_launch"]
                                 if (kernel_sources_hash() == TRAFFIC_CAPTURE["sources_sha256_16"]
                                     and R == TRAFFIC_CAPTURE["replicas"]
                                     and all(shape[k] == TRAFFIC_CAPTURE[k]
                                             for k in ("threads", "cluster")))
                                 else None),
                     "traffic_unit": "DRAM bytes per launch (ncu capture)",
                     "kernel": "pr_persistent<float>",
                     "bytes_per_hop": bytes_per_hop,
                     # the strict lower bound: the eps read-modify-write alone
                     # (2 s N bytes per hop, the two table reads counted as free)
                     "bytes_per_hop_strict": N * 2 * 4,
                     "frac_strict": achieved / 2 / smem_peak,
                     "peak_source": "measured: shared-memory 32-bit read-modify-write "
                                    "microbenchmark over all SMs (cg_microbench kind 0)",
                     # the eps-update phase alone (the bandwidth-bound step):
                     # algorithmic bytes over each CTA's update-phase clock
                     # cycles (clock64 of thread 0) against one SM's share of
                     # the measured peak; the one-replica figure is filled in
                     # below (fp32_single.update_phase.frac)
                     "update_phase_frac_batched": (
                         (hops * bytes_per_hop / (cyc_upd / (clk["sm_mhz"] * 1e6)))
                         / (smem_peak / sms) if clk and cyc_upd else None),
                     "update_phase_frac_one_replica": None,
                     "end_to_end_note": "frac covers the whole kernel, whose time is "
                                        "mostly the rejection phase at T=0.01"},
        # the rejection phase: evaluated labels per second against the
        # measured rate of the kernels' own Philox generator (every label
        # costs one block); "frac" over the whole launch time, "phase_frac"
        # over the share of the CTAs' cycles spent in label rounds
        "rejection_roofline": rejection_roofline(evaluated, sum(run_ms) * 1e-3, cyc_rej,
                                                 cyc_upd, philox_peak),
        # the refresh as a whole (error reset and the three FFT passes)
        # against the measured HBM copy rate
        "refresh_roofline": refresh_roofline(N, R, statistics.mean(ref_ms)),
        "phase_split": {"refresh_ms_per_step": statistics.mean(ref_ms),
                        "run_ms_per_step": statistics.mean(run_ms),
                        "update_cycles_frac": cyc_upd / max(1, cyc_upd + cyc_rej),
                        "max_eps_err_last_refresh": max_err},
        # per step: one persistent launch per L, then the refresh: error reset
        # and three FFT passes
        "gpu_launches": args.steps * (1 + 4),
        "clocks": clk,
        "peaks_measured": {"barrier_us_by_ctas": {str(c): v for c, v in barrier_us.items()},
                           "smem_rmw32_GBps": smem_peak / 1e9, "dadd_per_s": dadd_peak,
                           "philox_blocks_per_s": philox_peak},
        "wall_s_timed": t_wall,
    }
    # M sweep of the same relaxed batch: one refresh period of hops per M,
    # the persistent launch timed with events (M changes which labels are
    # drawn, not the chain's law)
    if not args.no_m_sweep:
        sweep = {}
        for Ms in (1024, 4096, 16384, 65536):
            o0 = [B.cg_observables(sysm.h, k) for k in range(R)]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            with torch.cuda.stream(st):
                ev[0].record(st)
                B.cg_run_async(sysm.h, HOPS_PER_STEP, Ms)
                ev[1].record(st)
                B.cg_refresh_async(sysm.h)
            assert B.cg_sync(sysm.h) == B.CG_OK
            o1 = [B.cg_observables(sysm.h, k) for k in range(R)]
            dt = ev[0].elapsed_time(ev[1]) * 1e-3
            d = {f: sum(b[f] - a[f] for a, b in zip(o0, o1)) for f in ("hops", "attempts",
                                                                          "evaluated")}
            sweep[str(Ms)] = {"hops_per_s": d["hops"] / dt, "attempts_per_s": d["attempts"] / dt,
                              "labels_evaluated_per_s": d["evaluated"] / dt}
        result["m_sweep"] = sweep
    # the relaxed batch state, the starting point of the end-to-end measurement
    snapshot = None if args.no_e2e else {
        g: sysm.read_group(g) for g in range(B.cg_num_groups(sysm.h))}
    sysm.close()

    # the plain binary64 form of the same workload (one replica, bit-exact with
    # the serial chain) and the binary32 form of one replica, both after the
    # same relaxation as the batched chains
    if args.fp64_hops > 0:
        relax = args.relax_steps * HOPS_PER_STEP
        for key, prec, hops in (("fp64_form", B.CG_FP64, args.fp64_hops),
                                ("fp32_single", B.CG_FP32, 4 * args.fp64_hops)):
            s1 = B.System(replicas_for(rank, 1), precision=prec, device=local,
                          refresh_every=HOPS_PER_STEP if prec == B.CG_FP32 else 0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            with torch.cuda.stream(s1.stream):
                B.cg_run_async(s1.h, relax, args.M)
                B.cg_sync(s1.h)
                o0 = B.cg_observables(s1.h, 0)
                ev[0].record(s1.stream)
                B.cg_run_async(s1.h, hops, args.M)
                ev[1].record(s1.stream)
                B.cg_sync(s1.h)
            o1 = B.cg_observables(s1.h, 0)
            dt = ev[0].elapsed_time(ev[1]) * 1e-3
            dh, da = o1["hops"] - o0["hops"], o1["attempts"] - o0["attempts"]
            result[key] = {"hops_per_s": dh / dt, "attempts_per_s": da / dt, "replicas": 1,
                           "hops": dh, "acceptance": dh / max(1, da),
                           "state": f"after {relax} hops from the random start"}
            if prec == B.CG_FP32 and clk:
                # eps-update phase of one replica alone on its SM: algorithmic
                # bytes over the update-phase time (SM clock cycles of the
                # update, thread 0's clock64) against one SM's share of the
                # measured shared-memory peak
                cyc = o1["cycles_update"] - o0["cycles_update"]
                t_upd = cyc / (clk["sm_mhz"] * 1e6)
                bw = dh * bytes_per_hop / t_upd
                per_sm = smem_peak / sms
                result[key]["update_phase"] = {
                    "achieved_GBps": bw / 1e9, "peak_per_sm_GBps": per_sm / 1e9,
                    "frac": bw / per_sm, "update_time_frac": cyc / max(
                        1, cyc + o1["cycles_reject"] - o0["cycles_reject"])}
                result["roofline"]["update_phase_frac_one_replica"] = bw / per_sm
            s1.close()
        # the binary64 form batched (one replica per SM) and one binary64
        # replica over an 8-CTA cluster (its update spread over 8 SMs' FP64
        # units); both bit-exact with the serial chain
        for key, R64, csize in (("fp64_batched", sms, 0), ("fp64_cluster8", 1, 8)):
            s1 = B.System(replicas_for(rank, R64), precision=B.CG_FP64, device=local,
                          cluster_size=csize)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            hops = args.fp64_hops if R64 > 1 else 4 * args.fp64_hops
            with torch.cuda.stream(s1.stream):
                B.cg_run_async(s1.h, relax, args.M)
                B.cg_sync(s1.h)
                o0 = [B.cg_observables(s1.h, k) for k in range(R64)]
                ev[0].record(s1.stream)
                B.cg_run_async(s1.h, hops, args.M)
                ev[1].record(s1.stream)
                B.cg_sync(s1.h)
            o1 = [B.cg_observables(s1.h, k) for k in range(R64)]
            dt = ev[0].elapsed_time(ev[1]) * 1e-3
            dh = sum(b["hops"] - a["hops"] for a, b in zip(o0, o1))
            da = sum(b["attempts"] - a["attempts"] for a, b in zip(o0, o1))
            sh = B.cg_group_shape(s1.h, 0)
            result[key] = {"hops_per_s": dh / dt, "attempts_per_s": da / dt, "replicas": R64,
                           "hops_per_replica": hops, "acceptance": dh / max(1, da),
                           "threads": sh["threads"], "cluster": sh["cluster"],
                           "state": f"after {relax} hops from the random start"}
            s1.close()
        result["fp64_form"]["update_bound_dadd_per_hop"] = 2 * N
        result["fp64_form"]["dadd_peak_per_s"] = dadd_peak
        result["fp32_batched_over_fp64_form"] = result["value"] / result["fp64_form"]["hops_per_s"]
        result["fp32_batched_over_fp64_batched"] = (result["value"]
                                                    / result["fp64_batched"]["hops_per_s"])
        result["fp64_cluster8"]["over_one_cta"] = (result["fp64_cluster8"]["hops_per_s"]
                                                   / result["fp64_form"]["hops_per_s"])
        result["fp64_cluster8"]["roofline"] = cluster_roofline(
            replicas_for(rank, 1), result["fp64_cluster8"]["hops_per_s"], 8, smem_peak, sms, "fp64")

    # binary32 form (with its binary64 refresh) against the binary64 form on
    # the same disorder samples: paired differences of the observables
    if args.obs_samples > 0 and rank == 0:
        result["fp32_vs_fp64_observables"] = observable_check(args, B, local)

    # the mixed-L batch and the cluster-sized lattice (not the headline
    # workload): throughput of their own launch paths
    if not args.no_other_configs and rank == 0:
        result["other_configs"] = other_configs(args, B, local, smem_peak=smem_peak, sms=sms,
                                                barrier_us=barrier_us)

    # sigma(t) relaxation at L=256: binary32 form against the binary64 form
    if args.sigma_hops > 0 and not args.no_other_configs and rank == 0:
        from paper_1407_5026_gb300 import sigma as S
        result["sigma_L256_fp32_vs_fp64"] = S.compare_forms_l256(B, local, args.sigma_hops)

    # sigma(t) relaxation of the L=64 configuration at T = 0.02, 0.05, 0.1
    # and its Eq. 4 scaling variables (the plateau sigma_0 per T)
    if args.sigma_l64_hops > 0 and not args.no_other_configs and rank == 0:
        result["sigma_L64_rescaling"] = sigma_l64_summary(B, local, args.sigma_l64_hops)

    # end to end through the C ABI with host buffers: upload the whole batch
    # state (occupations, binary32 eps, counters) from pinned host memory, run
    # one step, read it back; beside it the variant that moves the chain state
    # only (occupations, counters) and rebuilds eps from it on the device
    if not args.no_e2e:
        result["e2e"] = e2e(args, B, reps, local, snapshot, with_eps=True)
        result["e2e_chain_state_only"] = e2e(args, B, reps, local, snapshot)

    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.M,
                                              args.relax_steps * HOPS_PER_STEP)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def observable_check(args, B, local):
    """Runs the same obs_samples disorder replicas of the workload in binary32
    (refresh every 1024 hops) and in binary64 from their common random start
    for obs_hops hops; returns per observable the mean paired difference, its
    standard error and z = mean / SE, and the largest eps error any binary32
    replica saw at its refreshes."""
    import math
    import numpy as np
    reps = replicas_for(0, args.obs_samples)
    out = {}
    vals = {}
    for key, prec in (("fp32", B.CG_FP32), ("fp64", B.CG_FP64)):
        s = B.System(reps, precision=prec, device=local,
                     refresh_every=HOPS_PER_STEP if prec == B.CG_FP32 else 0)
        s.run(args.obs_hops, args.M)
        obs = [s.observables(k) for k in range(len(reps))]
        vals[key] = np.array([[o["energy_per_site"], o["P"], o["acceptance"]] for o in obs])
        if prec == B.CG_FP32:
            out["max_eps_err"] = max(o["max_eps_err_last_refresh"] for o in obs)
        s.close()
    d = vals["fp32"] - vals["fp64"]
    n = len(reps)
    for col, name in enumerate(("E_per_site", "P", "acceptance")):
        mean = float(d[:, col].mean())
        se = float(d[:, col].std(ddof=1) / math.sqrt(n))
        out[name] = {"fp64_mean": float(vals["fp64"][:, col].mean()),
                     "mean_diff": mean, "se": se, "z": (mean / se) if se > 0 else 0.0}
    out["samples"] = n
    out["hops"] = args.obs_hops
    out["start"] = "the random initial configuration of each replica, identical in both forms"
    return out


def rejection_roofline(evaluated, run_s, cyc_rej, cyc_upd, philox_peak):
    rate = evaluated / run_s
    share = cyc_rej / max(1, cyc_rej + cyc_upd)
    return {"bound": "alu", "achieved": rate / 1e9, "peak": philox_peak / 1e9,
            "unit": "G labels/s", "frac": rate / philox_peak,
            "phase_achieved": rate / share / 1e9, "phase_frac": rate / share / philox_peak,
            "rejection_cycle_share": share,
            "peak_source": "measured: Philox-4x32-10 blocks/s of the PR kernels' label "
                           "generator on all SMs (cg_microbench kind 3)",
            "kernel": "pr_persistent<float>"}


def refresh_roofline(N, R, ms):
    """The FFT refresh's bytes per replica and refresh: the occupation bits
    (N/8), four sweeps of its half of the complex transform buffer (4 x 4 N:
    written by the first pass, read and written by the second, read by the
    third), half of DFT(g)/N (2 N, one read per replica pair), phi (8 N) and
    eps read and written (8 N), against the measured HBM copy rate."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    if "hbm_gbs" in peaks:
        peak, src = float(peaks["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    else:
        peak, src = 6800.0, "of fallback (6.8 TB/s)"
    per_replica = N / 8.0 + 16.0 * N + 2.0 * N + 8.0 * N + 8.0 * N
    achieved = per_replica * R / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": src,
            "kernel": "fft_pass_kernel x 3 (+ error reset)",
            "bytes_per_refresh": per_replica * R}


def shape_of(B, h, g, tuned):
    sh = B.cg_group_shape(h, g)
    if not tuned:
        sh.pop("M")        # the group's own M applies only to runs with M = 0
    return sh


def cluster_roofline(reps, hops_per_s, cluster, smem_peak, sms, precision):
    """The eps update's algorithmic shared-memory bytes per second (16 N B
    per hop in binary32, 32 N in binary64) against the measured
    shared-memory peak of the SMs the launch occupies (one CTA per SM); N =
    L^2 on the square lattice, L^3 on the cubic one."""
    N = reps[0]["L"] ** (3 if reps[0].get("dim") == 3 else 2)
    per_hop = (16 if precision == "fp32" else 32) * N
    used = min(sms, len(reps) * cluster)
    peak = smem_peak * used / sms
    achieved = hops_per_s * per_hop
    return {"bound": "smem", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
            "frac": achieved / peak, "sms_used": used, "bytes_per_hop": per_hop}


def random_roofline(reps, hops_per_s):
    """The random-site update's HBM roofline: a hop reads rows j and i of the
    binary64 coupling matrix G (16 N bytes; G of a box past L ~ 32 is far
    larger than L2), against the measured HBM copy bandwidth."""
    N = reps[0]["L"] ** 2
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peak = float(json.load(f)["hbm_gbs"])
    ach = hops_per_s * 16.0 * N / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_hop": 16 * N, "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
            "note": "G-row bytes of the eps update only; the labels' partner lookups add "
                    "latency-bound gathers"}


def other_configs(args, B, local, only=None, smem_peak=None, sms=None, barrier_us=None):
    """Throughput of the other batch configurations: 256 replicas with L
    drawn from {32, 48, 64, 96} (one launch per L on concurrent streams,
    replayed as a CUDA graph, CTA size and M from the autotuner, an FFT
    refresh per same-L group every 1024 hops), 16 replicas of L=256 whose eps is split over a
    thread-block cluster (refresh every 4096 hops), 152 replicas of the
    32 x 32 x 32 cubic lattice (FFT refresh every 1024 hops), 38 replicas of
    the 48^3 lattice on 4-CTA clusters (eps split by z-planes), 304 replicas
    of L=64 with and
    without two-electron hops (a fifth of the labels proposing a pair), 19
    replicas of the 64^3 lattice on 8-CTA clusters (1/r of the update indexed
    by r^2), and
    152 binary64 replicas of L=64 (and of L=32) with sites at random
    positions against the L=64 replicas on the lattice, one random-site
    replica of L=128 on one CTA and on an 8-CTA cluster, and 16 random-site
    replicas of L=192 (eps of 36,864 sites: past one CTA) on autotuned
    clusters.  Each is timed with CUDA events over hops that follow a
    relaxation from the random start."""
    import torch
    from paper_1407_5026_gb300 import workloads as W
    out = {}
    for name, wl, relax, hops, graph, tune, forced, dflt in (
            ("mixed_L32-96_R256_T0.03", W.mixed_batch(), 8192, 4096, 1, True, 0, True),
            ("L256_T0.02_R16_cluster", W.l256(), 65536, 16384, 0, True, 0, True),
            # the same replicas on forced 4-CTA clusters without the
            # autotuner's trial launches (profiling with --config only)
            ("L256_T0.02_R16_cluster4", W.l256(), 65536, 4096, 0, False, 4, False),
            ("cubic_L32_T0.05_R152", W.cubic(), 4096, 4096, 0, False, 0, True),
            ("cubic_L48_T0.05_R38_cluster4", W.cubic(R=38, L=48), 2048, 2048, 0, False, 0, True),
            # 8 replicas of 32^3 on one CTA each and on forced 4-CTA clusters
            # (small cases for profiling the cubic cluster kernel; --config only)
            ("cubic_L32_T0.05_R8", W.cubic(R=8), 4096, 2048, 0, False, 0, False),
            ("cubic_L32_T0.05_R8_cluster4", W.cubic(R=8), 4096, 2048, 0, False, 4, False),
            # 19 replicas of 64^3 on 8-CTA clusters (152 SMs), the update
            # reading 1/r by r^2 (the folded table fits beside no eps share)
            ("cubic_L64_T0.05_R19_cluster8", W.cubic(R=19, L=64), 2048, 4096, 0, False, 0,
             True),
            ("pairs_L64_T0.05_R304_p0.2", W.pairs(), 4096, 4096, 0, False, 0, True),
            ("single_L64_T0.05_R304", W.pairs(pair_frac=0.0), 4096, 4096, 0, False, 0, True),
            ("random_L64_T0.05_R152_fp64", W.random_sites(), 2048, 2048, 0, False, 0, True),
            ("random_L32_T0.05_R152_fp64", W.random_sites(L=32), 2048, 2048, 0, False, 0, True),
            ("lattice_L64_T0.05_R152_fp64", W.random_sites(lattice=True), 2048, 2048, 0, False,
             0, True),
            ("random_L128_T0.05_R1_fp64", W.random_sites(R=1, L=128), 4096, 4096, 0, False, 0,
             True),
            ("random_L128_T0.05_R1_fp64_cluster8", W.random_sites(R=1, L=128), 4096, 4096, 0,
             False, 8, True),
            ("random_L192_T0.05_R16_fp64_cluster", W.random_sites(R=16, L=192), 2048, 4096, 0,
             True, 0, True)):
        if only is not None and name != only:
            continue
        if not dflt and only is None:
            continue
        reps = [r.as_dict() for r in wl.replicas]
        pair = {k: wl.extra[k] for k in ("pair_frac", "pair_rmax") if wl.extra.get("pair_frac")}
        prec = B.CG_FP64 if wl.precision == "fp64" else B.CG_FP32
        # a random-site box holds an 8 N^2-byte coupling matrix per replica
        # (174 GB for 16 replicas of L=192): the library allocates it and
        # frees it at close, outside torch's cache
        big = any(r.get("sites") and r["L"] > 128 for r in reps)
        s = B.System(reps, precision=prec, refresh_every=wl.refresh_every,
                     use_graph=graph, device=local, cluster_size=forced,
                     torch_memory=not big, **pair)
        s.run(relax, wl.M)
        if tune:
            B.cg_autotune(s.h, 256)
        M = 0 if tune else wl.M
        o0 = [B.cg_observables(s.h, k) for k in range(len(reps))]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(s.stream):
            ev[0].record(s.stream)
            B.cg_run_async(s.h, hops, M)
            ev[1].record(s.stream)
            B.cg_sync(s.h)
        o1 = [B.cg_observables(s.h, k) for k in range(len(reps))]
        dt = ev[0].elapsed_time(ev[1]) * 1e-3
        dh = sum(b["hops"] - a["hops"] for a, b in zip(o0, o1))
        da = sum(b["attempts"] - a["attempts"] for a, b in zip(o0, o1))
        out[name] = {"hops_per_s": dh / dt, "attempts_per_s": da / dt, "acceptance": dh / max(1, da),
                     "replicas": len(reps), "hops_per_replica": hops, "relaxed_hops": relax,
                     "M": "autotuned per L" if tune else wl.M,
                     "groups": [shape_of(B, s.h, g, tune) for g in range(B.cg_num_groups(s.h))],
                     "max_eps_err": max(o["max_eps_err_last_refresh"] for o in o1),
                     "graph": bool(graph),
                     # share of the kernels' SM cycles spent in the eps update
                     # (the rest: label rounds), from the per-replica phase
                     # clocks over the timed hops
                     "update_cycle_share": update_share(o0, o1)}
        cl = max(g["cluster"] for g in out[name]["groups"])
        if reps[0].get("sites"):
            out[name]["roofline"] = random_roofline(reps, out[name]["hops_per_s"])
        elif cl > 1 and smem_peak and sms:
            out[name]["roofline"] = cluster_roofline(reps, out[name]["hops_per_s"], cl,
                                                     smem_peak, sms, wl.precision)
            if barrier_us:
                # a hop of one replica against the measured cluster barrier
                # (each chunk and each hop ends in one)
                out[name]["roofline"]["hop_us"] = len(reps) / out[name]["hops_per_s"] * 1e6
                out[name]["roofline"]["cluster_barrier_us"] = barrier_us.get(cl)
        if pair:
            out[name].update(pair)
            out[name]["pair_hops_share"] = pair_share(B, s, reps, wl.M)
        s.close()
    return out


def update_share(o0, o1):
    upd = sum(b["cycles_update"] - a["cycles_update"] for a, b in zip(o0, o1))
    rej = sum(b["cycles_reject"] - a["cycles_reject"] for a, b in zip(o0, o1))
    return round(upd / max(1, upd + rej), 4)


def sigma_l64_summary(B, local, hops):
    """sigma(t) of the L=64 relaxation configuration (8 disorder seeds per T)
    and its Eq. 4 variables: per T the acceptance, sigma_0 (slope of P over
    the last decade of time), the run's last time, tau = 1/(sigma_0 T^2) and
    the windows (t, x = t sigma_0 T^2, y = sigma / sigma_0)."""
    from paper_1407_5026_gb300 import sigma as S
    r = S.relaxation_curves(B, device=local, hops=hops)
    out = {}
    for T, v in r.items():
        out[str(T)] = {"acceptance": v["acceptance"], "sigma0": v["sigma0"], "t_end": v["t_end"],
                       "tau": 1.0 / (v["sigma0"] * T * T) if v["sigma0"] > 0 else None,
                       "t": [round(x, 4) for x in v["t"]],
                       "x": [float(f"{x:.4g}") for x in v["x"]],
                       "y": [round(y, 4) for y in v["y"]]}
    return out


def pair_share(B, s, reps, M, hops=64):
    """Share of two-electron hops among the next `hops` hops of every
    replica (from their hop logs)."""
    import numpy as np
    rc, log = s.run_logged(hops, M)
    return float(np.mean(log["k"] != 0xFFFFFFFF))


def e2e(args, B, reps, local, snapshot, with_eps=False):
    """The same metric through the public C ABI with host buffers: every step
    uploads the batch's chain state from pinned host memory with
    cg_write_group_state, runs one step (cg_run + cg_refresh) and reads the
    state back into the same pinned buffers with cg_read_group_state.  The
    chain state is the occupations and the counters; eps is derived from the
    occupations, so after the upload cg_refresh rebuilds it on the device
    (0.15 ms for the batch) instead of copying 20 MB each way.  with_eps:
    binary32 eps also goes both ways (no rebuild).  The batch starts from
    the relaxed state the device-timed steps ended in (same seeds, so the
    same disorder)."""
    import numpy as np
    import torch
    R = len(reps)
    N = WORKLOAD["L"] ** 2
    words = (N + 31) // 32
    sysm = B.System(reps, precision=B.CG_FP32, refresh_every=0, block_threads=args.threads,
                    device=local)
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
    groups = list(range(B.cg_num_groups(sysm.h)))
    bufs = {}
    for g in groups:
        # pinned copies of the timed run's final (relaxed) state of the group
        cnt = len(B.cg_group_replicas(sysm.h, g))
        occ, eps = pin((cnt, words), torch.int32).view(np.uint32), pin((cnt, N), torch.float32)
        occ[:] = snapshot[g][0]
        eps[:] = snapshot[g][1]
        bufs[g] = [occ, eps, snapshot[g][2].copy()]
    steps = max(3, min(args.steps, 8))
    M_run = args.M
    if not args.no_tune:
        B.cg_autotune(sysm.h, HOPS_PER_STEP)           # the headline batch's cached shape
        M_run = 0
    B.cg_run(sysm.h, HOPS_PER_STEP, M_run)             # warm
    torch.cuda.synchronize()
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_initialized() else 1
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    hops = attempts = 0
    for _ in range(steps):
        for g in groups:
            sysm.write_group(g, occ=bufs[g][0], eps=bufs[g][1] if with_eps else None,
                             counters=bufs[g][2])
        if not with_eps:
            B.cg_refresh_async(sysm.h)                 # eps from the uploaded occupations
        B.cg_run_async(sysm.h, HOPS_PER_STEP, M_run)
        B.cg_refresh_async(sysm.h)
        B.cg_sync(sysm.h)
        for g in groups:
            _, _, c = sysm.read_group(g, occ=bufs[g][0], eps=bufs[g][1] if with_eps else False)
            hops += int((c["hops"] - bufs[g][2]["hops"]).sum())
            attempts += int((c["attempts"] - bufs[g][2]["attempts"]).sum())
            bufs[g][2] = c
    dt = time.perf_counter() - t0
    sysm.close()
    # the whole job: every rank's hops over the slowest rank's time
    dt, hops, attempts = combine_ranks(dt, hops, attempts, device=f"cuda:{local}")
    # per replica and step: bitmask words (and binary32 eps) each way; the
    # 112-byte device counter block read once and written once by the group
    # write (which keeps the library's own fields) and read once by the read
    e = 4 * N if with_eps else 0
    h2d = ws * R * (4 * words + e + 112)                # the whole job's bytes
    d2h = ws * R * (4 * words + e + 2 * 112)
    note = ("per step: cg_write_group_state (occupations, counters) + cg_refresh (eps rebuilt "
            "from the uploaded occupations) + cg_run + cg_refresh + cg_read_group_state "
            "(occupations, counters) for the whole batch from/to pinned host buffers"
            if not with_eps else
            "per step: cg_write_group_state (occupations, binary32 eps, counters) + cg_run + "
            "cg_refresh + cg_read_group_state (the same) from/to pinned host buffers")
    # attempts/s beside hops/s: these steps come later in the chains'
    # relaxation than the device-timed ones (acceptance slowly falling)
    return {"value": hops / dt, "unit": "hops/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "attempts_per_s": attempts / dt,
            "acceptance": hops / max(1, attempts), "note": note}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
