#!/usr/bin/env python
"""Sampled paths/s of one CentRA sample-and-cover round on GB300.

A step is one pass of the whole hot path over one batch: draw M pairs,
count shortest paths, walk one uniform shortest path per pair, append the
hyper-edges, build the node -> sample incidence, greedyCover(k), the t sign
vectors and AMCERA numerators, and the FP64 bounds / stopping test (one round
of Algorithm 1 at m = M).  Every step uses a fresh job with its own seed so no
step reuses another's samples.  The graph (synthetic R-MAT scale 18 LCC,
stand-in for the paper's SNAP graphs) stays resident in HBM.

Prints one JSON line.  `--impl reference` times the CPU oracle (the plain
single-threaded C statement of the method) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_03651_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "rmat18": ("R-MAT scale 18 (262,144 ids), edge factor 16, (.57,.19,.19,.05), undirected, dedup, no self-loops, LCC",
               I.rmat18_lcc),
    "ba2000": ("Barabasi-Albert n=2000, 4 edges per new node, seed 1", I.ba_2000),
    "grid2048": ("2048x2048 4-neighbour grid, 1% of edges rewired, undirected", I.grid2048_rewired),
    "rmat22d": ("R-MAT scale 22, edge factor 16, directed, dedup, no self-loops", I.rmat22_directed),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat18", choices=sorted(WORKLOADS))
    ap.add_argument("--m", type=int, default=65536, help="pairs sampled per step")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttc", action="store_true", help="skip the time-to-certified block of the round mode")
    ap.add_argument("--serial-round", action="store_true",
                    help="greedyCover and the AMCERA one after the other instead of side by side")
    ap.add_argument("--mode", default="round", choices=["round", "batch", "serve", "tsweep", "schedule"],
                    help="round: one Algorithm-1 round per step (default); batch: time to certified eps of the "
                         "64-job BA workload, one job at a time vs batched; serve: Poisson request stream; "
                         "tsweep: fixed-m rounds over the number t of Rademacher vectors (SD bound and time); "
                         "schedule: time to certified eps with the doubling and the paper's sample schedule")
    ap.add_argument("--sampler", type=int, default=0, help="0 bidirectional (default), 1 bit-parallel waves")
    ap.add_argument("--bidir-budget", type=float, default=0, help="bytes of bidirectional workspace (0: default)")
    ap.add_argument("--bidir-queue", type=int, default=0, help="nodes per ball / cone list (0: default)")
    ap.add_argument("--bidir-warps", type=int, default=-1,
                    help="1: warp searches handed to the CTA when they outgrow a warp; 0: whole-CTA searches; "
                         "2: escalated searches in a second launch (-1: library default)")
    ap.add_argument("--bidir-table", type=int, default=-2,
                    help="node-table entries per CTA (-1: sized for L2, 0: none; -2: library default)")
    ap.add_argument("--space", type=int, default=0, help="hyper-edge space: 0 set betweenness, 1 kappa-path, 2 triangle")
    ap.add_argument("--kappa", type=int, default=8, help="path bound of the kappa-path space")
    ap.add_argument("--tsweep-m", type=int, default=500000)
    ap.add_argument("--tsweep-t", default="1,10,50,100,250,500")
    ap.add_argument("--tsweep-k", type=int, default=50)
    ap.add_argument("--schedule-eps", default="0.1,0.05")
    ap.add_argument("--schedule-k", default="", help="values of k for the schedule mode (default: the workload's)")
    ap.add_argument("--schedule-plans", default="",
                    help="schedule:rule pairs for the schedule mode, e.g. 'predict:centra,doubling:centra' "
                         "(default: all five)")
    ap.add_argument("--batch-jobs", type=int, default=64)
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-eps", default="0.01,0.005")
    ap.add_argument("--serve-workers", type=int, default=8)
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self, interval_ms: int = 50):
        """Starts sampling and returns once the first sample is in (at most 3 s), so that the
        timed region that follows is sampled from its start."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t_begin: float | None = None, t_end: float | None = None):
        """Median SM clock and the throttle reasons seen; with t_begin/t_end (perf_counter), only
        samples taken inside that window (plus one interval) count, if there are any."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        lines = self.lines
        if t_begin is not None and t_end is not None:
            inside = [x for x in lines if t_begin <= x[0] <= t_end + 0.06]
            lines = inside or lines
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# kernel class -> (committed ncu summary, source file whose hash it records)
DRAM_PROFILES = {"expand_pull": ("expand_pull_dram.md", "sampler.cu"), "bidir": ("bidir_dram.md", "bidir.cu")}


def dram_traffic(kernel_class: str, workload: str, pairs_per_step: int):
    """DRAM bytes per launch of `kernel_class` from the committed ncu summary, or None when there
    is none for the class, its source changed since the counters were taken, or the summary's
    launch is another workload or step size (the traffic of a launch depends on both)."""
    import hashlib
    if kernel_class not in DRAM_PROFILES:
        return None
    prof = os.path.join(ROOT, "profiles", DRAM_PROFILES[kernel_class][0])
    src = os.path.join(ROOT, "paper_2306_03651_gb300", "csrc", DRAM_PROFILES[kernel_class][1])
    try:
        kv = {}
        for line in open(prof):
            if ":" in line and not line.startswith(("|", "#", " ")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if (kv.get("kernel_class") == kernel_class and kv.get("source_sha256_16") == sha
                and kv.get("workload") == workload and int(kv.get("pairs_per_step", -1)) == pairs_per_step):
            return float(kv["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


# ----------------------------------------------------------------- replicas
def rank_seed(rank: int) -> int:
    """Seed of rank `rank`'s replica: distinct per rank, so replicas draw disjoint sample streams."""
    return 1_000_003 * (rank + 1)


def reduce_max(value: float, device) -> float:
    """Max of `value` over all ranks (the slowest replica times the job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- gpu arm
SPACE = {"space": 0, "kappa": 0}  # hyper-edge space of the round mode (set from the arguments)


SERIAL_ROUND = {"on": False}  # --serial-round: greedyCover, then the AMCERA, as two calls


def cover_and_mcera(job, k):
    """greedyCover and the AMCERA of the round: side by side on two streams (one call), or, with
    --serial-round, one after the other (two calls); the outputs are the same."""
    if SERIAL_ROUND["on"]:
        S, cov = job.greedy_cover(k)
        Rnum, Wnum, b = job.mcera(k)
        return S, cov, Rnum, Wnum, b
    return job.cover_and_mcera(k)


def gpu_step(P, graph, wl, M, seed, events=None):
    """One Algorithm-1 round on a new job: sample M pairs, greedyCover and the AMCERA, bounds.
    `events` (start, end), when given, are recorded on the job's stream around the round alone:
    the job's creation, its statistics and its release are not part of it."""
    job = P.Job(graph, seed, wl.t, space=SPACE["space"], kappa=SPACE["kappa"])
    job.set_timing(True)
    if events:
        events[0].record()
    job.sample(M)
    S, cov, Rnum, Wnum, b = cover_and_mcera(job, wl.k)
    stop, bd = P.bounds(cov, M, int(Rnum.sum()), wl.t, Wnum, b, wl.eps, wl.delta, 1)
    if events:
        events[1].record()
    SAMPLER_INFO.append(job.sampler_info())
    st = job.stats()
    job.close()
    return st, (S, cov, Rnum, Wnum, b, stop, bd)


SAMPLER_INFO = []  # per step: how the bidirectional sampler handled the pairs


def merge_stats(acc, st):
    for k, v in st.items():
        a = acc.setdefault(k, dict(launches=0, ms=0.0, timed=0, units=0))
        for f in a:
            a[f] += v[f]


def apply_sampler_args(P, graph, args):
    """Sampler choice and workspace limits as defaults for every job on the graph."""
    if args.sampler:
        graph.set_param(P.PARAM_SAMPLER, args.sampler)
    if args.bidir_budget:
        graph.set_param(P.PARAM_BIDIR_BUDGET, args.bidir_budget)
    if args.bidir_queue:
        graph.set_param(P.PARAM_BIDIR_QUEUE, args.bidir_queue)
    if args.bidir_table != -2:
        graph.set_param(P.PARAM_BIDIR_TABLE, args.bidir_table)
    if args.bidir_warps >= 0:
        graph.set_param(P.PARAM_BIDIR_WARPS, args.bidir_warps)


def time_to_certified(P, graph, g, wl, args):
    """Algorithm 1 to certification on the resident graph (cen_run) under the doubling and the
    predicting schedule, and the same through the public API with host buffers: the graph
    uploaded from pinned host memory inside the timed region and the results read back."""
    import torch
    plans = (("doubling", P.SCHEDULE_DOUBLING), ("predicting", P.SCHEDULE_EXTRAPOLATE))
    P.run(graph, wl.k, 0.1, wl.delta, wl.t, 999, m0=1000)  # warm-up (workspaces, pools)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    t_begin = time.perf_counter()
    out = {"workload": args.workload, "k": wl.k, "eps": wl.eps, "delta": wl.delta, "t": wl.t, "m0": 1000,
           "seed": wl.seed, "how": "host wall clock around cen_run (device synchronized on both sides)"}
    for name, sched in plans:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.run(graph, wl.k, wl.eps, wl.delta, wl.t, wl.seed, m0=1000, schedule=sched, alpha=1.2)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out[name] = {"seconds": el, "status": "certified" if r["status"] == P.OK else "not certified",
                     "m_final": r["m_final"], "rounds": r["rounds"], "covered": r["covered"],
                     "C": float(r["log"][-1][6]) if r["rounds"] else None}
    off_h = torch.from_numpy(g.off).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    e2e = {"h2d_bytes": int(g.off.nbytes + g.col.nbytes)}
    for name, sched in plans:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gg = P.Graph(g.n, off_h.numpy(), col_h.numpy(), g.directed)
        apply_sampler_args(P, gg, args)
        r = P.run(gg, wl.k, wl.eps, wl.delta, wl.t, wl.seed, m0=1000, schedule=sched, alpha=1.2)
        gg.close()
        torch.cuda.synchronize()
        e2e[name] = {"seconds": time.perf_counter() - t0, "m_final": r["m_final"],
                     "same_as_resident": r["m_final"] == out[name]["m_final"] and r["covered"] == out[name]["covered"]}
    out["e2e_host_buffers"] = e2e
    out["clocks"] = clocks.stop(t_begin, time.perf_counter())
    return out


def run_gpu(args, rank, world):
    import torch
    import paper_2306_03651_gb300 as P

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    desc, make = WORKLOADS[args.workload]
    wl = make()
    g = wl.graph
    graph = P.Graph.of(g)
    apply_sampler_args(P, graph, args)
    SPACE.update(space=args.space, kappa=args.kappa if args.space == 1 else 0)
    M = args.m
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2 (129 MB)
    seed0 = rank_seed(rank)
    for w in range(args.warmup):
        gpu_step(P, graph, wl, M, seed0 + w)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    stats, times = {}, []
    t0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st, _ = gpu_step(P, graph, wl, M, seed0 + 1000 + s, (a, b))
        b.synchronize()
        times.append(a.elapsed_time(b))
        merge_stats(stats, st)
    torch.cuda.synchronize()
    t_done = time.perf_counter()
    wall = t_done - t0
    clk = clocks.stop(t0, t_done)
    total_ms = float(sum(times))
    if world > 1:
        total_ms = reduce_max(total_ms, "cuda")
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = world * M * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers: graph upload from
    # pinned memory, the round, results back to the host
    e2e = None
    if not args.no_e2e:
        off_h = torch.from_numpy(g.off).pin_memory()
        col_h = torch.from_numpy(g.col).pin_memory()
        torch.cuda.synchronize()
        et = []
        for s in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            gg = P.Graph(g.n, off_h.numpy(), col_h.numpy(), g.directed)
            apply_sampler_args(P, gg, args)
            job = P.Job(gg, seed0 + 2000 + s, wl.t, space=SPACE["space"], kappa=SPACE["kappa"])
            job.sample(M)
            S, cov, Rnum, Wnum, b = cover_and_mcera(job, wl.k)
            P.bounds(cov, M, int(Rnum.sum()), wl.t, Wnum, b, wl.eps, wl.delta, 1)
            job.close()
            gg.close()
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t1)
        e_tot = sum(et)
        if world > 1:
            e_tot = reduce_max(e_tot, "cuda")
        e2e = {"value": world * M * args.steps / e_tot, "unit": "paths/s",
               "h2d_bytes_per_step": int(g.off.nbytes + g.col.nbytes),
               "d2h_bytes_per_step": int(4 * wl.k + 8 * wl.t + 8 + 4 + 8 + 4)}

    # roofline: the kernel class with the most device time; its algorithmic
    # bytes are counted by the kernels themselves, per unit of their class
    import json as _json
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            pk = _json.load(f)
        peak, peak_src = float(pk["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    byte_classes = ("bidir", "expand_pull", "expand_push", "level_finalize", "cone", "cone_sigma", "walk")
    dom = max(stats, key=lambda k: stats[k]["ms"])
    roof = None
    if stats[dom]["ms"] > 0:
        avg_ms = stats[dom]["ms"] / max(stats[dom]["timed"], 1)
        per_launch_bytes = stats[dom]["units"] / max(stats[dom]["launches"], 1)
        achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9 if dom in byte_classes else None
        counted = sum(stats[k]["units"] for k in byte_classes if k in stats)
        sampler_default = (not args.sampler and not args.bidir_budget and not args.bidir_queue
                           and args.bidir_table == -2 and args.bidir_warps < 0)
        traffic = dram_traffic(dom, args.workload, M) if sampler_default and args.space == 0 else None
        ratio = (f"DRAM traffic {traffic / per_launch_bytes:.2f}x the counted bytes, from an ncu DRAM capture"
                 if traffic and per_launch_bytes else "DRAM traffic not profiled for this source and workload")
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                "avg_launch_ms": avg_ms, "launches": stats[dom]["launches"],
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "note": ("one launch samples the whole step; the kernel is bound by the latency of dependent L2 "
                         f"accesses ({ratio})"
                         if dom == "bidir" else
                         "per-launch event times of concurrent wave pipelines include sharing the GPU"),
                "aggregate_counted_GBps": counted / (total_ms / 1e3) / 1e9}
    launches = int(sum(v["launches"] for v in stats.values()))
    ttc = None
    if rank == 0 and not args.no_ttc and args.space == 0 and args.workload in ("rmat18", "ba2000"):
        ttc = time_to_certified(P, graph, g, wl, args)
    out = {
        "metric": "sampled paths/s" if args.space == 0 else "sampled hyper-edges/s", "value": value,
        "unit": "paths/s" if args.space == 0 else "hyper-edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}; one Algorithm-1 round per step at m={M} pairs, "
                               f"k={wl.k}, t={wl.t}, eps={wl.eps}, delta={wl.delta}",
                   "n": g.n, "arcs": g.nnz, "pairs_per_step": M, "l2": "flushed (256 MB write) between steps",
                   "timed": "the round (sample, greedyCover and AMCERA, bounds) on a job created just before it",
                   "space": ["set betweenness", f"kappa-path (kappa={args.kappa})", "triangle"][args.space],
                   "parallelism": f"replicas x{world}",
                   "round": ("greedyCover then AMCERA (two calls)" if args.serial_round
                             else "greedyCover and AMCERA side by side (cen_cover_and_mcera)")},
        "e2e": e2e, "gpu_launches": launches, "clocks": clk, "roofline": roof, "time_to_certified": ttc,
        "sampler": SAMPLER_INFO[-1] if SAMPLER_INFO else None,
        "wall_s": wall,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "units": v["units"]}
                    for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]},
    }
    return out, wl


# ---------------------------------------------------------------- cpu oracle
def oracle_rate(wl, seconds: float, seed: int = 424242):
    """The oracle (single thread) on a bounded sample: pairs, walks, greedyCover, AMCERA, bounds."""
    import oracle as O

    og = O.Graph.of(wl.graph)
    probe = O.Job(og, seed, wl.t)
    t0 = time.perf_counter()
    probe.sample(4)
    per = max((time.perf_counter() - t0) / 4, 1e-6)
    count = int(max(8, min(200000, seconds / per)))
    job = O.Job(og, seed + 1, wl.t)
    t0 = time.perf_counter()
    job.sample(count)
    S, cov = job.greedy_cover(wl.k)
    Rn, Wn, b = job.mcera(wl.k)
    O.bounds(cov, count, int(Rn.sum()), wl.t, Wn, b, wl.eps, wl.delta, 1)
    el = time.perf_counter() - t0
    LAST_ORACLE_WORK[:] = [count, *job.work().tolist()]
    return count / el, count, el


# the oracle's work tallies of the last oracle_rate sample: pairs, then nodes reached
# before the target's level, arcs scanned out of them, in-arcs scanned by the walks,
# path members written
LAST_ORACLE_WORK: list = []


def oracle_bytes_per_pair(work) -> float:
    """Algorithmic bytes per pair of the forward search the oracle states (SURVEY-style
    count): 16 per node reached before the target's level (distance and count), 16 per arc
    scanned out of those levels (the arc, the head's distance check and count add), 16 per
    in-arc the walk scans, 4 per member written."""
    pairs, nodes, arcs, walk, members = work
    return (16 * nodes + 16 * arcs + 16 * walk + 4 * members) / max(pairs, 1)


def run_batch_mode(args):
    """Time to certified eps of the batched workload, every job to certification:
    the plain form (one job at a time, each sample searched by a whole CTA), the same
    sequence with the library's default sampler settings, and the batched form
    (cen_run_batch: jobs concurrently on worker streams) with the default settings and
    with settings autotuned per graph beforehand (tuning timed apart); all four give
    identical results."""
    import torch
    import paper_2306_03651_gb300 as P
    from paper_2306_03651_gb300 import tune

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    params = I.ba_batch_params(args.batch_jobs)
    graphs = [P.Graph.of(I.ba(p["n"], p["d"], p["graph_seed"])) for p in params]
    jobs = [dict(graph=g, k=p["k"], eps=0.01, delta=0.1, t=32, seed=p["job_seed"], m_cap=1 << 27)
            for g, p in zip(graphs, params)]
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for g in graphs:
        g.set_param(P.PARAM_BIDIR_WARPS, 0)
    t0 = time.perf_counter()
    plain = P.run_batch(jobs, nworkers=1)
    t_plain = time.perf_counter() - t0
    for g in graphs:
        g.set_param(P.PARAM_BIDIR_WARPS, -1)
    t0 = time.perf_counter()
    plain_default = P.run_batch(jobs, nworkers=1)
    t_plain_default = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = P.run_batch(jobs, nworkers=args.batch_workers)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    # probes of a full round: smaller ones time one wave of the warp kernel, not its throughput
    tuned = [tune.autotune(g, t=32, probe_pairs=65536, grid=tune.SAMPLER_GRID)["best"] for g in graphs]
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched_tuned = P.run_batch(jobs, nworkers=args.batch_workers)
    t_batch_tuned = time.perf_counter() - t0
    clk = clocks.stop()

    def same(a, b):
        return all(x["S"].tolist() == y["S"].tolist() and x["m_final"] == y["m_final"] and x["covered"] == y["covered"]
                   and np.array_equal(x["log"], y["log"]) for x, y in zip(a, b))
    samples = sum(r["m_final"] for r in batched)
    print(json.dumps({
        "metric": "time to certified eps (s)", "value": t_batch, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.batch_jobs} BA jobs, n log-uniform in [1e4, 5e5], 2-8 edges per node, "
                               f"k in {{10,50,100}}, eps=0.01, delta=0.1, t=32, m0=1000 doubling",
                   "batched_workers": args.batch_workers},
        "plain_s": t_plain, "plain_default_s": t_plain_default, "batched_s": t_batch,
        "batched_tuned_s": t_batch_tuned, "tuning_s": t_tune,
        "speedup": t_plain / t_batch, "speedup_vs_plain_default": t_plain_default / t_batch,
        "identical_results": same(plain, batched) and same(plain_default, batched) and same(batched_tuned, batched),
        "certified": sum(1 for r in batched if r["status"] == P.OK), "samples_total": samples,
        "paths_per_s_batched": samples / t_batch, "paths_per_s_plain": samples / t_plain,
        "tuned_warp_searches": sum(1 for c in tuned if c["bidir_warps"] == 1), "clocks": clk,
    }))


def run_tsweep_mode(args):
    """Fixed-m rounds over t (the shape of the paper's Sec. 6 experiment on the impact of t:
    m = 5e5, delta = 0.05, k = 50): per t, the AMCERA, the SD bound eta and the time of one
    round (sample, greedyCover, AMCERA, bounds), each step a fresh job with its own seed."""
    import torch
    import paper_2306_03651_gb300 as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    desc, make = WORKLOADS[args.workload]
    wl = make()
    graph = P.Graph.of(wl.graph)
    M, k, delta = args.tsweep_m, args.tsweep_k, 0.05
    ts = [int(x) for x in args.tsweep_t.split(",")]
    rows = []
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for t in ts:
        times, etas = [], []
        for step in range(-1, max(args.steps, 1)):  # step -1 is the warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            job = P.Job(graph, 9000 + 97 * t + step, t)
            job.sample(M)
            S, cov = job.greedy_cover(k)
            Rnum, Wnum, b = job.mcera(k)
            stop, bd = P.bounds(cov, M, int(Rnum.sum()), t, Wnum, b, 0.05, delta, 1)
            job.close()
            el = time.perf_counter() - t0
            bd["etaU"] = P.bounds_hedge(cov, M, wl.graph.n, k, 0.05, delta, 1)[1]["etaU"]
            if step >= 0:
                times.append(el)
                etas.append(bd)
        rows.append({"t": t, "round_s": statistics.median(times),
                     "eta": statistics.median(e["eta"] for e in etas),
                     "eta_union_bound": statistics.median(e["etaU"] for e in etas),
                     "amcera": statistics.median(e["A"] for e in etas),
                     "R": statistics.median(e["R"] for e in etas),
                     "C": statistics.median(e["C"] for e in etas)})
    clk = clocks.stop()
    print(json.dumps({
        "metric": "fixed-m round time over t", "value": rows[-1]["round_s"], "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "m": M, "k": k, "delta": delta, "t": ts},
        "rows": rows, "clocks": clk,
    }))


def run_schedule_mode(args):
    """Time to certified eps of one job per sample schedule (doubling from m0 = 1000; the paper's
    growth by 1.2 plus the optimistic guess; that plus the predicted size) and stopping rule
    (CentRA's AMCERA bounds; HEDGE-P's union bound), the shape of the paper's progressive-sampling
    comparison."""
    import torch
    import paper_2306_03651_gb300 as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    desc, make = WORKLOADS[args.workload]
    wl = make()
    graph = P.Graph.of(wl.graph)
    P.run(graph, wl.k, 0.2, wl.delta, wl.t, 1, m0=1000)  # warm-up
    rows = []
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    plans = (("doubling", P.SCHEDULE_DOUBLING, "centra", P.RULE_CENTRA),
             ("paper", P.SCHEDULE_PAPER, "centra", P.RULE_CENTRA),
             ("predict", P.SCHEDULE_EXTRAPOLATE, "centra", P.RULE_CENTRA),
             ("doubling", P.SCHEDULE_DOUBLING, "hedge_p", P.RULE_HEDGE_P),
             ("predict", P.SCHEDULE_EXTRAPOLATE, "hedge_p", P.RULE_HEDGE_P))
    if args.schedule_plans:
        want = [tuple(x.split(":")) for x in args.schedule_plans.split(",")]
        plans = tuple(p for w in want for p in plans if (p[0], p[2]) == w)
        if len(plans) != len(want):
            raise SystemExit(f"--schedule-plans: unknown plan in {args.schedule_plans!r}")
    ks = [int(x) for x in args.schedule_k.split(",")] if args.schedule_k else [wl.k]
    for k, eps in ((k, float(e)) for k in ks for e in args.schedule_eps.split(",")):
        for name, sched, rname, rule in plans:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = P.run(graph, k, eps, wl.delta, wl.t, wl.seed, m0=1000, m_cap=1 << 30, schedule=sched,
                      alpha=1.2, rule=rule)
            el = time.perf_counter() - t0
            rows.append({"k": k, "eps": eps, "schedule": name, "rule": rname, "status": r["status"], "seconds": el,
                         "rounds": r["rounds"], "m_final": r["m_final"],
                         "C": float(r["log"][-1][6]) if r["rounds"] else None,
                         "eta": float(r["log"][-1][13]) if r["rounds"] else None})
    clk = clocks.stop()
    print(json.dumps({
        "metric": "time to certified eps (s)", "value": rows[-1]["seconds"], "unit": "s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "k": ks, "t": wl.t, "delta": wl.delta},
        "rows": rows, "clocks": clk,
    }))


def run_serve_mode(args):
    """Poisson request stream on device-resident graphs (BA 2000, R-MAT 18 LCC, 8 of
    the batched BA graphs); capacity first (all requests at t=0), then arrival
    rates 0.5 / 0.7 / 0.9 x capacity."""
    import torch
    import paper_2306_03651_gb300 as P
    from paper_2306_03651_gb300 import serve as SV

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    graphs = {"ba2000": P.Graph.of(I.ba(2000, 4, 1)), "rmat18": P.Graph.of(I.rmat18_lcc().graph)}
    for j, p in enumerate(I.ba_batch_params(8)):
        graphs[f"ba{j}"] = P.Graph.of(I.ba(p["n"], p["d"], p["graph_seed"]))
    names = sorted(graphs)
    eps_list = [float(x) for x in args.serve_eps.split(",")]
    rng = np.random.default_rng(11)
    N = args.serve_requests
    reqs = [SV.Request(rid=i, graph=names[int(rng.integers(len(names)))], k=int(rng.integers(10, 201)),
                       eps=float(eps_list[int(rng.integers(len(eps_list)))]), delta=0.1, t=10, seed=5000 + i,
                       m_cap=1 << 27) for i in range(N)]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    srv = SV.Server(graphs, workers=args.serve_workers)
    res = srv.serve(reqs)
    cap = SV.summarize(res)
    cap.update(peak_running=srv.peak_running, round_waits=srv.waits)
    rows = {"capacity": cap}
    print(json.dumps({"pass": "capacity", **cap}), file=sys.stderr, flush=True)
    for frac in (0.5, 0.7, 0.9):
        arr = SV.poisson_arrivals(N, frac * cap["jobs_per_s"], seed=int(frac * 100))
        for r, a in zip(reqs, arr):
            r.arrival_s = a
        srv = SV.Server(graphs, workers=args.serve_workers)
        res = srv.serve(reqs)
        rows[f"lambda_{frac}"] = SV.summarize(res)
        rows[f"lambda_{frac}"].update(peak_running=srv.peak_running, round_waits=srv.waits)
        print(json.dumps({"pass": f"lambda_{frac}", **rows[f"lambda_{frac}"]}), file=sys.stderr, flush=True)
    clk = clocks.stop()
    print(json.dumps({
        "metric": "jobs/s", "value": rows["lambda_0.9"]["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": f"{N} requests, graphs {names}, k ~ U[10,200], eps in {eps_list}, delta=0.1, t=10",
                   "workers": args.serve_workers},
        "p50_latency_s": rows["lambda_0.9"]["p50_latency_s"], "p99_latency_s": rows["lambda_0.9"]["p99_latency_s"],
        "runs": rows, "clocks": clk,
    }))


def _oracle_shard(payload):
    """Worker of the sharded oracle: samples ids [a, b) of one job (CPU, one core)."""
    n, off, col, directed, seed, t, a, b = payload
    import oracle as O
    g = O.Graph(n, off, col, directed)
    job = O.Job(g, seed, t)
    t0 = time.perf_counter()
    job.sample_from(a, b - a)
    return time.perf_counter() - t0


def oracle_sharded_rate(wl, count: int, procs: int, seed: int = 424243):
    """The oracle's sampling split by sample index over `procs` processes (spawned): pairs/s
    over the slowest shard.  Context for the single-core baseline; samples are identical."""
    import multiprocessing as mp
    g = wl.graph
    bounds = [count * p // procs for p in range(procs + 1)]
    payloads = [(g.n, g.off, g.col, g.directed, seed, wl.t, bounds[p], bounds[p + 1]) for p in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        times = pool.map(_oracle_shard, payloads)
    return count / max(times), max(times)


def main():
    args = parse()
    SERIAL_ROUND["on"] = args.serial_round
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.mode == "batch":
        if rank == 0:
            run_batch_mode(args)
        return
    if args.mode == "serve":
        if rank == 0:
            run_serve_mode(args)
        return
    if args.mode == "tsweep":
        if rank == 0:
            run_tsweep_mode(args)
        return
    if args.mode == "schedule":
        if rank == 0:
            run_schedule_mode(args)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        desc, make = WORKLOADS[args.workload]
        wl = make()
        for _ in range(args.warmup):
            oracle_rate(wl, min(2.0, args.cpu_seconds / 4))
        rates, counts, els = [], [], []
        for _ in range(args.steps):
            r, c, e = oracle_rate(wl, args.cpu_seconds / max(args.steps, 1))
            rates.append(r)
            counts.append(c)
            els.append(e)
        tot = sum(counts) / sum(els)
        sample = f"{sum(counts)} pairs over {args.steps} steps ({sum(els):.1f} s), each step one oracle round"
        print(json.dumps({
            "impl": "reference", "metric": "sampled paths/s", "value": tot, "unit": "paths/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(els) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}; one Algorithm-1 round per step (bounded sample), "
                                   f"k={wl.k}, t={wl.t}", "n": wl.graph.n, "arcs": wl.graph.nnz},
            "cpu_baseline": {"value": tot, "unit": "paths/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": tot, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, wl = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            r, c, e = oracle_rate(wl, args.cpu_seconds)
            out["cpu_baseline"] = {"value": r, "unit": "paths/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{c} pairs of the same workload, one oracle round ({e:.1f} s)"}
            roof = out.get("roofline")
            if roof and roof.get("kernel") == "bidir" and roof.get("launches") == out["steps"] and args.space == 0:
                # the oracle's count of a forward search's bytes against the kernel's own count
                bpp = oracle_bytes_per_pair(LAST_ORACLE_WORK)
                counted = roof["algorithmic_bytes_per_launch"] / args.m
                roof["oracle_basis"] = {"forward_bytes_per_pair": bpp, "counted_bytes_per_pair": counted,
                                        "work_ratio": bpp / counted, "pairs_sampled": LAST_ORACLE_WORK[0],
                                        "note": "bytes a forward search to d(s,t) needs per pair (the oracle's "
                                                "tallies on its sample) against the bytes the bidirectional "
                                                "kernel counts per pair; the roofline uses the kernel's count"}
            procs = os.cpu_count() or 1
            if procs > 1:
                cnt = max(procs, int(r * args.cpu_seconds / 2) * procs)
                rs, el = oracle_sharded_rate(wl, cnt, procs)
                out["cpu_baseline_sharded"] = {"value": rs, "unit": "paths/s", "cores": procs, "kind": "oracle",
                                               "sample": f"{cnt} pairs split by sample index over {procs} "
                                                         f"processes (slowest shard {el:.1f} s), sampling only"}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
