#!/usr/bin/env python
"""Benchmark of GB300 sort-based matching (one JSON line on stdout).

Workload (default): d = 1, N = 1e6 extents (500k subscriptions + 500k
updates), float32 starts uniform in [0, 1e6), equal length alpha * L / N with
alpha = 100 (the paper's Section 5 methodology), enumerate mode: the full
sorted (sub, upd) pair list, K ~ 5e7 pairs.  One step = one ddm_match call
(key build, radix sort, sweep scan, counts, offsets, emission, segment sort)
with inputs and output resident in HBM; a 256 MiB buffer is written between
timed steps so that the 8 MB of inputs never start in L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (serial Algorithm 4 in C) on the host
cores instead, each step a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (its own seed):
the matching of independent instances needs no exchange, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
REF_SAMPLE_SUBS = 250_000   # oracle sample: first 250k subscriptions x all updates (d = 1)
REF_SAMPLE_SUBS_ND = 20_000  # d > 1: the dimension-0 candidates per subscription are many more


def ref_sample_subs(args) -> int:
    return REF_SAMPLE_SUBS if args.d == 1 else REF_SAMPLE_SUBS_ND


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--alpha", type=float, default=100.0)
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=1, help="dimensions (1 = the headline workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--incremental-only", action="store_true",
                    help="only the session change-report section (a profiling case)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(args, rank: int):
    d = getattr(args, "d", 1)
    if d == 1:
        return synth.large_1d(args.alpha, replica=rank, N=args.N)
    return synth.large_nd(d, args.alpha, replica=rank, N=args.N)


def workload_name(args):
    return (f"d={getattr(args, 'd', 1)}, N={args.N:.0e} ({args.N // 2} subs + "
            f"{args.N - args.N // 2} upds), alpha={args.alpha:g}, enumerate (sorted pair list)")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(reg, seconds: float, nsub: int = REF_SAMPLE_SUBS):
    import oracle
    sample = synth.Regions(reg.sub_lo[:, :nsub].copy(),
                           reg.sub_hi[:, :nsub].copy(), reg.upd_lo, reg.upd_hi)
    times, K = [], 0
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end or not times:
        t0 = time.perf_counter()
        K = len(oracle.sbm(sample))
        times.append(time.perf_counter() - t0)
    return {"value": K / statistics.mean(times), "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nsub} subscriptions x all {reg.m} updates of the "
                      f"same workload (K={K}), serial C Algorithm 4 + pair sort, "
                      f"{len(times)} runs, host cpu_count={os.cpu_count()}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    reg = workload(args, 0)
    nsub = ref_sample_subs(args)
    sample = synth.Regions(reg.sub_lo[:, :nsub].copy(),
                           reg.sub_hi[:, :nsub].copy(), reg.upd_lo, reg.upd_hi)
    for _ in range(args.warmup):
        oracle.sbm(sample)
    times, K = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        K = len(oracle.sbm(sample))
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = K * args.steps / total
    line = {"impl": "reference", "metric": "matched pairs/s", "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args) + f"; each step a bounded sample: first "
                                                         f"{nsub} subscriptions",
                       "N": args.N, "d": args.d, "alpha": args.alpha, "K_sample": K},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {nsub} subscriptions x all updates"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched(ctx, dev, steps: int = 3):
    """4096 independent instances (d=2, alpha=1, N_i log-uniform in [1e2, 1e5]) in one
    ddm_match_batch call, against 4096 plain ddm_match calls on the same stream."""
    import torch
    regs = synth.batch_instances(num=4096, d=2)
    insts = [[torch.from_numpy(a).to(dev) for a in (r.sub_lo, r.sub_hi, r.upd_lo, r.upd_hi)]
             for r in regs]
    pack = ctx.pack_batch(insts)
    K, offs = ctx.match_batch_packed(pack)
    out = torch.empty((max(K, 1), 2), dtype=torch.int32, device=dev)
    ctx.match_batch_packed(pack, out[:K])
    stream = torch.cuda.current_stream(dev)
    gpu_ms, wall = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        ctx.match_batch_packed(pack, out[:K], offs)
        e1.record(stream)
        torch.cuda.synchronize()
        wall.append(time.perf_counter() - t0)
        gpu_ms.append(e0.elapsed_time(e1))
    packs = [ctx.pack(*i) for i in insts]
    views = [out[int(offs[b]):int(offs[b + 1])] for b in range(len(insts))]
    for b in range(len(insts)):
        ctx.match_packed(packs[b], views[b])
    torch.cuda.synchronize()
    plain = []
    for _ in range(2):
        t0 = time.perf_counter()
        for b in range(len(insts)):
            ctx.match_packed(packs[b], views[b])
        torch.cuda.synchronize()
        plain.append(time.perf_counter() - t0)
    bw, pw = min(wall), min(plain)
    return {"workload": "4096 instances, d=2, alpha=1, N_i log-uniform in [1e2, 1e5]",
            "regions": int(sum(r.n + r.m for r in regs)), "K": K,
            "batched_gpu_ms": min(gpu_ms), "batched_wall_ms": 1e3 * bw,
            "batched_pairs_per_s": K / bw, "plain_wall_ms": 1e3 * pw, "plain_pairs_per_s": K / pw,
            "speedup_vs_plain": pw / bw}


def bench_baselines(ctx, dev, reps: int = 5):
    """The paper's matchers on the same GPU: Sort-Based (this library's path),
    Interval-Tree (Algorithm 3), Grid-Based (Section 2, the library's grid
    size) and Brute-Force (Algorithm 2), all writing the full sorted pair
    list, at N = 1e5 (brute force is O(n m))."""
    import torch
    out = {}
    for d, alpha in ((1, 100.0), (2, 1.0)):
        N = 100_000
        reg = synth.large_1d(alpha, N=N) if d == 1 else synth.large_nd(d, alpha, N=N)
        t = [torch.from_numpy(a).to(dev) for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]
        K = ctx.count(*t)
        buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        res = {"workload": f"d={d}, N={N:.0e}, alpha={alpha:g}, sorted pair list", "K": K}
        calls = {"sbm": lambda: ctx.match_into(buf[:K], *t),
                 "itm": lambda: ctx.match_itm(*t, cap=K),
                 "grid": lambda: ctx.match_grid(*t, cap=K),
                 "bruteforce": lambda: ctx.match_bruteforce(*t, cap=K)}
        for name, fn in calls.items():
            fn()
            ms = []
            for _ in range(reps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            res[f"{name}_ms"] = statistics.median(ms)
            res[f"{name}_pairs_per_s"] = K / (res[f"{name}_ms"] * 1e-3)
        res["bruteforce_over_sbm"] = res["bruteforce_ms"] / res["sbm_ms"]
        res["itm_over_sbm"] = res["itm_ms"] / res["sbm_ms"]
        res["grid_over_sbm"] = res["grid_ms"] / res["sbm_ms"]
        res["grid_cells"] = ctx.last_grid
        out[f"d{d}"] = res
    return out


def bench_incremental(args, dev, steps: int = 10, warmup: int = 3):
    """The headline workload as a session: every timestep drifts the extents by
    N(0, 0.01 side) and reports only the pairs that appeared or disappeared
    (ddm_session_emit_delta, which counts the timestep itself), against count +
    full emission of the same timestep; both also measured with their result
    delivered to pinned host memory (what a consumer off the GPU receives)."""
    import torch
    import paper_1703_06680_gb300 as ddm
    reg = workload(args, 0)
    t_in = [torch.from_numpy(a).to(dev) for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]
    sess = ddm.Session(*t_in)
    sigma = 0.01 * synth.side_for(args.alpha, args.N, args.d)
    K0 = sess.count()
    big = torch.empty((max(K0, 1), 2), dtype=torch.int32, device=dev)
    sess.emit_delta(big[:K0], big[:0])       # first report: every pair
    cap = max(K0 // 8, 4096)
    add_b = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    rem_b = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    host = torch.empty((max(K0, 1) + 4096, 2), dtype=torch.int32).pin_memory()
    stream = torch.cuda.current_stream(dev)
    step = 0

    def timed(fn, n):
        nonlocal step
        tot = 0.0
        out = None
        for _ in range(n):
            sess.drift(1703, step, sigma)
            step += 1
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / max(n, 1), out

    def report(to_host=False):
        # One library call: the report counts the drifted timestep itself (a report
        # needs no K first; the full emission below needs K to size its output).
        a, r = sess.emit_delta(add_b, rem_b)
        if to_host:
            host[:len(a)].copy_(a, non_blocking=True)
            host[len(a):len(a) + len(r)].copy_(r, non_blocking=True)
        return sess.K, len(a), len(r)

    def full(to_host=False):
        K = sess.count()
        sess.emit(big[:K])
        if to_host:
            host[:K].copy_(big[:K], non_blocking=True)
        return K, K, 0

    timed(report, warmup)
    report_ms, (K, na, nr) = timed(report, steps)
    report_host_ms, _ = timed(lambda: report(True), steps)
    timed(full, warmup)
    full_ms, _ = timed(full, steps)
    full_host_ms, _ = timed(lambda: full(True), steps)
    sess.close()
    return {"workload": workload_name(args) + ", session with drift N(0, 0.01 side) per step",
            "steps": steps, "warmup": warmup, "K": K, "report_ms": report_ms,
            "full_emit_ms": full_ms, "report_to_host_ms": report_host_ms,
            "full_emit_to_host_ms": full_host_ms, "added_per_step": na, "removed_per_step": nr,
            "report_bytes_per_step": 8 * (na + nr), "full_bytes_per_step": 8 * K}


def bench_served(dev, requests: int = 96, slots: int = 4, load: float = 0.8):
    """64 simulations (N log-uniform in [1e3, 1e6], d and alpha uniform), drift between
    timesteps, Poisson arrivals at `load` x the plain path's measured capacity."""
    import torch

    from paper_1703_06680_gb300.serve import Server, Simulation, latency_summary, run_plain
    cfg = synth.served_simulations(64)
    regs = [synth.simulation_regions(c) for c in cfg]
    sig = [0.1 * synth.side_for(c["alpha"], c["N"], c["d"]) for c in cfg]

    def make_sims():
        return [Simulation(k, [torch.from_numpy(a).to(dev) for a in
                               (r.sub_lo, r.sub_hi, r.upd_lo, r.upd_hi)], cfg[k]["seed"] ^ 0xD41F7,
                           sig[k]) for k, r in enumerate(regs)]

    rng = np.random.default_rng(64)
    order = rng.integers(0, 64, size=requests)
    from paper_1703_06680_gb300.serve import Request

    # 1) plain capacity: all requests queued at once, one at a time
    sims = make_sims()
    reqs = [Request(sim=int(k), arrival=0.0) for k in order]
    cap_wall = run_plain(sims, reqs)
    capacity = requests / cap_wall
    plain_sat_pairs = sum(r.K for r in reqs) / cap_wall
    for s_ in sims:
        s_.close()

    # 1b) served capacity: the same requests all queued at once, with `slots`
    # slots (overlap) and with one slot (count reuse and resident state, no overlap)
    def saturated(nslots):
        sims = make_sims()
        server = Server(sims, slots=nslots)
        t0 = time.perf_counter()
        sat = [server.submit(int(k), arrival=t0) for k in order]
        for r in sat:
            r.done.wait(600)
        wall_ = max(r.finish for r in sat) - t0
        server.close()
        for s_ in sims:
            s_.close()
        return sum(r.K for r in sat) / wall_, wall_

    served_sat_pairs, sat_wall = saturated(slots)
    served1_sat_pairs, sat1_wall = saturated(1)
    def served_at(offsets, nslots):
        sims = make_sims()
        server = Server(sims, slots=nslots)
        t0 = time.perf_counter()
        sreqs = []
        for k, off in zip(order, offsets):
            now = time.perf_counter() - t0
            if off > now:
                time.sleep(off - now)
            sreqs.append(server.submit(int(k), arrival=t0 + off))
        for r in sreqs:
            r.done.wait(600)
        served_wall = max(r.finish for r in sreqs) - t0
        server.close()
        for s_ in sims:
            s_.close()
        return latency_summary(sreqs, served_wall)

    def at_load(lf: float):
        rate_ = lf * capacity
        offsets = np.cumsum(np.random.default_rng(int(lf * 1000)).exponential(1.0 / rate_,
                                                                              size=requests))
        # served: continuous batching at the offered load, and the one-slot server
        srv = served_at(offsets, slots)
        srv1 = served_at(offsets, 1)
        # plain at the same offered load (queueing included)
        sims = make_sims()
        t0 = time.perf_counter()
        preqs = [Request(sim=int(k), arrival=t0 + off) for k, off in zip(order, offsets)]
        run_plain(sims, preqs)
        plain_wall = max(r.finish for r in preqs) - t0
        pln = latency_summary(preqs, plain_wall)
        for s_ in sims:
            s_.close()
        return rate_, srv, srv1, pln

    sweep = {}
    for lf in (0.5, 0.8, 1.0):
        r_, srv, srv1, pln = at_load(lf)
        sweep[str(lf)] = {"offered_rps": r_, "served_p50_ms": srv["p50_ms"],
                          "served_p99_ms": srv["p99_ms"],
                          "served_1slot_p50_ms": srv1["p50_ms"],
                          "served_1slot_p99_ms": srv1["p99_ms"],
                          "plain_p50_ms": pln["p50_ms"], "plain_p99_ms": pln["p99_ms"],
                          "p99_speedup": pln["p99_ms"] / srv["p99_ms"] if srv["p99_ms"] else None}
        if lf == load:
            rate, served, plain = r_, srv, pln
    torch.cuda.empty_cache()
    return {"workload": "64 simulations, N log-uniform in [1e3, 1e6], d in {1,2,3}, "
                        "alpha in {0.01,1,100}, drift N(0, 0.1 side) per step, Poisson arrivals",
            "requests": requests, "slots": slots, "offered_load_vs_plain_capacity": load,
            "plain_capacity_rps": capacity, "offered_rps": rate, "served": served,
            "plain": plain,
            "plain_note": "one ddm_match per request on the session's resident coordinates, "
                          "buffer sized by the previous K (retry when it does not fit)",
            "saturated": {"plain_pairs_per_s": plain_sat_pairs, "served_pairs_per_s": served_sat_pairs,
                          "served_1slot_pairs_per_s": served1_sat_pairs,
                          "plain_rps": capacity, "served_rps": requests / sat_wall,
                          "served_1slot_rps": requests / sat1_wall,
                          "throughput_speedup": served_sat_pairs / plain_sat_pairs,
                          "overlap_speedup_vs_1slot": served_sat_pairs / served1_sat_pairs},
            "p99_speedup": plain["p99_ms"] / served["p99_ms"] if served["p99_ms"] else None,
            "load_sweep": sweep,
            "throughput_speedup": served["pairs_per_s"] / plain["pairs_per_s"]
            if plain["pairs_per_s"] else None}


def job_totals(t_ms: float, K: int, steps: int, e2e_s: float, e2e_steps: int, world: int, dev):
    """Whole-job figures over all ranks (weak scaling: every rank its own
    problem): the slowest rank's device time and end-to-end time, and the
    pairs of all ranks.  With world > 1 this reduces over the default process
    group (NCCL on the GPU machine; gloo with dev = cpu in the multi-rank tests)."""
    import torch
    import torch.distributed as dist
    times = torch.tensor([t_ms, e2e_s], dtype=torch.float64, device=dev)
    k_all = torch.tensor([float(K)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
        dist.all_reduce(k_all, op=dist.ReduceOp.SUM)
    t_max_s = float(times[0].item()) / 1e3
    e2e_max_s = float(times[1].item())
    pairs = float(k_all.item())
    return {"t_max_s": t_max_s, "pairs_all_ranks": pairs,
            "value": pairs * steps / t_max_s, "ms_per_step": 1e3 * t_max_s / steps,
            "e2e_value": pairs * e2e_steps / e2e_max_s}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1703_06680_gb300 as ddm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.incremental_only:
        print(json.dumps({"incremental": bench_incremental(args, dev)}), flush=True)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    reg = workload(args, rank)
    t_in = [torch.from_numpy(a).to(dev) for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]
    stream = torch.cuda.current_stream(dev)
    ctx = ddm.Context(local, stream=stream)
    K = ctx.count(*t_in)
    out = torch.empty((max(K, 1), 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        return ctx.match_into(out[:K], *t_in)

    # Warm-up steps with events at every stage boundary: they find the dominant
    # stage, the one the roofline reports.
    ctx.set_profiling(True)
    warm_sum = {}
    for _ in range(args.warmup):
        flush.fill_(1.0)
        assert step() == K
        for k, v in ctx.stats()["stage_ms"].items():
            warm_sum[k] = warm_sum.get(k, 0.0) + v
    top = max(warm_sum, key=warm_sum.get)
    # Timed steps: events only around the dominant stage (an event between two
    # kernels ends the programmatic-dependent-launch overlap there, so events at
    # every boundary would slow the step down).
    ctx.set_profiling(True, stage=ddm.STAGE_NAMES.index(top))
    top_sum = 0.0
    l0 = ctx.stats()["launches"]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))               # L2 flush, outside the timed events
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
        top_sum += ctx.stats()["stage_ms"][top]
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.stats()["launches"] - l0
    clocks = sampler.stop()
    # Stage breakdown: the same steps again, events at every stage boundary.
    ctx.set_profiling(True)
    stage_sum = {}
    for s in range(args.steps):
        flush.fill_(float(s))
        step()
        for k, v in ctx.stats()["stage_ms"].items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    ctx.set_profiling(False)
    t_ms = sum(a.elapsed_time(b) for a, b in ev)

    # End to end through the public API with HOST buffers (pinned), copies inside.
    host_in = [torch.from_numpy(a).pin_memory().numpy() for a in
               (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]
    host_out = torch.empty((max(K, 1), 2), dtype=torch.int32).pin_memory().numpy()
    e2e_steps = max(3, min(args.steps, 30))
    for _ in range(2):
        ctx.match_host(*host_in, out=host_out[:K])
    barrier()
    e2e_t = 0.0
    for _ in range(e2e_steps):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = ctx.match_host(*host_in, out=host_out[:K])
        e2e_t += time.perf_counter() - t0
    assert len(got) == K
    tot = job_totals(t_ms, K, args.steps, e2e_t, e2e_steps, world, dev)
    value, ms_step, e2e_value = tot["value"], tot["ms_per_step"], tot["e2e_value"]
    t_max_s = tot["t_max_s"]

    # Roofline of the dominant stage (per-stage CUDA events on the launching stream).
    stage_avg = {k: v / args.steps for k, v in stage_sum.items()}
    N, n, m = args.N, reg.n, reg.m
    E = 2 * N
    alg_bytes = {   # algorithmic bytes per launch of each stage (d = 1 window path)
        "keybuild": 8 * N + 16 * E,
        "radix_sort": 4 * 16 * E - 4 * E,
        # payloads read, one 16-byte rank record written per endpoint
        "sweep_scan": 4 * E + 16 * E,
        "counts": 12 * n,
        # both records read, count and offset written, 32-byte subscription and
        # 16-byte update rank entries scattered
        "offsets": 32 * N + 12 * n + 32 * n + 16 * m,
        # subscription entries read, candidates read (16 B) and packed (8 B)
        "emit_setup": 32 * n + 24 * m,
        "emit": 8 * K,
        "segsort": 8 * K,
    }
    hbm, peak_kind = peaks()
    top_ms = top_sum / args.steps        # measured inside the timed steps
    achieved = alg_bytes.get(top, 0) / (top_ms * 1e-3) / 1e9 if top_ms > 0 else 0.0
    traffic = None
    prof_txt = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof_txt):
        with open(prof_txt) as fh:
            traffic = json.load(fh).get(top)
    path_bytes = 8 * N * args.d + 8 * K
    line = {
        "metric": "matched pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "N": N, "d": args.d, "alpha": args.alpha, "K": K,
                   "seed": synth.seed_for(1 if args.d == 1 else 2, rank),
                   "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps"},
        "regions_per_s": N * world * args.steps / t_max_s,
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel_ms": top_ms},
        "path_roofline": {"bytes_alg": path_bytes, "achieved_gbs": path_bytes / (ms_step * 1e-3) / 1e9,
                          "frac": path_bytes / (ms_step * 1e-3) / 1e9 / hbm},
        "stages_ms": stage_avg,
        "stages_note": "per-stage events on every boundary, in a second pass of the same steps",
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": 4 * 2 * (n + m) * args.d,
                "d2h_bytes_per_step": 8 * K},
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    # The emission's store pattern without its filter (one warp per output
    # segment, segments of unrelated ids in flight together), measured here:
    # the ceiling that the emission's bandwidth is read against.
    if args.d == 1 and top == "emit" and n > 0 and K > 0:
        wp = {"segments": n, "mean_pairs": max(1, round(K / n))}
        for name, sc in (("scattered", True), ("sequential", False)):
            ms, nb = ctx.debug_write_pattern(n, wp["mean_pairs"], scattered=sc, reps=5)
            wp[name + "_gbs"] = nb / (ms * 1e-3) / 1e9
        line["write_pattern"] = wp
        line["roofline"]["pattern_ceiling_gbs"] = wp["scattered_gbs"]
        line["roofline"]["frac_of_pattern"] = achieved / wp["scattered_gbs"]
    if args.d > 1:
        # d > 1 is bound by the per-candidate filter: report the dimension-0
        # candidates (pairs that intersect in dimension 0, an exact d = 1 count of
        # the projection) resolved per second.
        K0 = ctx.count(*[t[:1] for t in t_in])
        line["candidates"] = {"dim0_candidates": K0,
                              "candidate_tests_per_s": K0 * world / t_max_s * args.steps}
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = bench_batched(ctx, dev)
        line["baselines"] = bench_baselines(ctx, dev)
    if rank == 0 and world == 1 and not args.no_served:
        line["served"] = bench_served(dev)
        line["incremental"] = bench_incremental(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(reg, args.cpu_seconds, ref_sample_subs(args))
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
