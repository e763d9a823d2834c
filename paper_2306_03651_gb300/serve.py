"""Continuous-batching request loop for CentRA jobs on device-resident graphs.

Requests (graph name, k, eps, delta, t, seed) arrive over time.  A request is
admitted as soon as a worker is free and the estimated device memory of its
first round fits in the HBM budget; admitted requests run Algorithm 1
concurrently, each on its own CUDA stream, so their kernels overlap on the GPU,
and each keeps its growing sample on the device across its progressive rounds.
Before each round a request reserves the memory of its grown sample, waiting
if the budget is short (the oldest running request never waits).  Finished
requests release their memory and worker at once, so waiting ones are
admitted mid-flight.  A request's result does not depend on what runs
beside it: samples, signs and picks are functions of (graph, seed, parameters).

Latency is arrival -> completion; the loop reports p50 / p99 latency and jobs/s.
"""
from __future__ import annotations

import ctypes
import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import cen as P


@dataclass
class Request:
    rid: int
    graph: str
    k: int
    eps: float
    delta: float
    t: int
    seed: int
    arrival_s: float = 0.0
    m0: int = 1000
    m_cap: int = 1 << 27


@dataclass
class Result:
    rid: int
    status: int
    S: np.ndarray
    covered: int
    m_final: int
    rounds: int
    log: np.ndarray
    arrival_s: float
    start_s: float
    end_s: float
    est_bytes: int
    error: str = ""  # the library's message when status is an error

    @property
    def latency_s(self) -> float:
        return self.end_s - self.arrival_s


def estimate_job_bytes(n: int, nnz: int, t: int, m_cap: int, avg_hyperedge: float = 8.0, levels: int = 16,
                       bidir_budget: int = 16 << 30, bidir_queue: int = 1 << 16, resident_ctas: int = 2432) -> int:
    """Upper estimate of one job's device memory (admission policy, not the method).

    Bidirectional sampler: one workspace per resident CTA (a large node table
    and as many path counts, H = 4 `bidir_queue` entries each, seven lists of
    `bidir_queue` entries, and a small table of at most 80 MiB over all CTAs),
    as many as fit in `bidir_budget`.  Wave workspace (the fallback): `levels` + 6 arrays
    of n*G words (G = wave words, at most 32 and at most 1 GB per array) and the
    initial cone-arc log (2 n G records of 24 bytes); sample store for m_cap
    samples: offsets, endpoints, distance, sign words and members (twice: samples
    and the incidence), plus the member arena; AMCERA table R[t+1][n] and greedy /
    incidence arrays.  `resident_ctas` is the sampler's CTAs in flight (16 per SM
    on a 152-SM GB300)."""
    qc = max(16, min(n, bidir_queue))
    h2 = 1024
    while h2 < 4 * qc:
        h2 *= 2
    per_slot = 16 * h2 + 7 * 4 * qc
    bidir = min(resident_ctas, max(1, bidir_budget // per_slot)) * per_slot + (80 << 20)
    G = 32
    while G > 1 and n * G * 8 > (1 << 30):
        G //= 2
    words = n * G
    wave = 8 * words * (levels + 6) + 24 * 2 * words
    nw = (t + 31) // 32
    store = m_cap * (8 + 12 + 4 * nw) + 3 * 4 * int(m_cap * avg_hyperedge)
    node = n * (4 * (t + 1) + 4 * 4 + 8)
    return int(bidir + wave + store + node)


def run_rounds(graph, req: Request, stream, reserve) -> dict:
    """Algorithm 1 for one request, one round at a time, as ``cen_run`` runs it with the
    doubling schedule and CentRA's rule: sample up to m_i, greedyCover beside the
    AMCERA, the FP64 bounds and the stopping test (Thm. 4.4, Alg. 1), then m_{i+1} = 2 m_i.
    ``reserve(m)`` is called before each round that grows the sample, with the new size,
    and may block until the server's memory budget has room for it."""
    job = P.Job(graph, req.seed, req.t, stream=stream)
    try:
        m_prev, m, i = 0, min(req.m0, req.m_cap), 0
        rows = []
        while True:
            i += 1
            reserve(m)
            job.sample(m - m_prev)
            S, cov, Rnum, Wnum, b = job.cover_and_mcera(req.k)
            Rsum = int(Rnum.sum())
            stop, bd = P.bounds(cov, m, Rsum, req.t, Wnum, b, req.eps, req.delta, i)
            rows.append([i, m, cov, Rsum, Wnum, b, bd["C"], bd["A"], bd["w"], bd["nu"], bd["xi"], bd["Rt"], bd["R"],
                         bd["eta"], float(stop), len(S)])
            if stop or 2 * m > req.m_cap:
                status = P.OK if stop else P.ENOTCERTIFIED
                break
            m_prev, m = m, 2 * m
        return dict(status=status, S=S, covered=cov, m_final=m, rounds=i, log=np.array(rows, np.float64))
    finally:
        job.close()


class Server:
    """Admission by HBM budget, one CUDA stream per worker, FIFO order.

    A request is admitted when a worker is free and the footprint of its first round
    fits the budget (or nothing runs).  Before each later round it reserves the
    footprint of the grown sample; if that does not fit, it waits for running requests
    to finish, except the oldest running request, which never waits, so the loop always
    progresses without preempting anyone (only that request's growth can take the total
    past the budget); no new request is admitted while one waits to grow.
    ``runner(graph, request, stream, reserve)`` runs one request
    (default: ``run_rounds`` on the library)."""

    def __init__(self, graphs: dict, workers: int = 8, hbm_budget_bytes: int | None = None, runner=None):
        import torch
        self.graphs = graphs
        self.workers = workers
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget_bytes = int(free * 0.8)
        self.budget = hbm_budget_bytes
        self.runner = runner or run_rounds
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self._cv = threading.Condition()
        self._queue: deque = deque()
        self._in_use = 0
        self._held: dict = {}      # rid -> bytes reserved
        self._running: list = []   # rids in admission order
        self._free_workers = list(range(workers))
        self._results: list[Result] = []
        self._t0 = 0.0
        self.peak_bytes = 0
        self.peak_running = 0
        self.waits = 0             # rounds that waited for memory
        self._blocked = 0          # running requests waiting to grow (new ones are not admitted meanwhile)

    def _est(self, r: Request, m: int) -> int:
        g = self.graphs[r.graph]
        return estimate_job_bytes(g.n, g.nnz, r.t, m)

    def _now(self) -> float:
        return time.perf_counter() - self._t0

    def _reserve(self, r: Request, m: int):
        """Grow r's reservation to the footprint of a sample of m; blocks while the budget
        is short, unless r is the oldest running request."""
        with self._cv:
            extra = self._est(r, m) - self._held[r.rid]
            if extra <= 0:
                return
            waited = False
            while self._in_use + extra > self.budget and self._running[0] != r.rid:
                if not waited:
                    waited = True
                    self._blocked += 1
                self._cv.wait(timeout=0.05)
            if waited:
                self.waits += 1
                self._blocked -= 1
            self._in_use += extra
            self._held[r.rid] += extra
            self.peak_bytes = max(self.peak_bytes, self._in_use)

    def _run_one(self, w: int, r: Request, arrival: float):
        g = self.graphs[r.graph]
        start = self._now()
        res = None
        try:
            out = self.runner(g, r, ctypes.c_void_p(self.streams[w].cuda_stream), lambda m: self._reserve(r, m))
            res = Result(r.rid, out["status"], out["S"], out["covered"], out["m_final"], out["rounds"], out["log"],
                         arrival, start, self._now(), self._held.get(r.rid, 0))
        except Exception as e:  # the request ends with its error status; its worker and bytes go back below
            res = Result(r.rid, int(getattr(e, "rc", P.ECUDA)), np.zeros(0, np.int32), 0, 0, 0,
                         np.zeros((0, len(P.LOG_COLS))), arrival, start, self._now(), self._held.get(r.rid, 0),
                         error=str(e))
        finally:
            with self._cv:
                if res is not None:
                    self._results.append(res)
                self._in_use -= self._held.pop(r.rid, 0)
                self._running.remove(r.rid)
                self._free_workers.append(w)
                self._cv.notify_all()

    def _dispatch(self, total: int):
        threads = []
        done = 0
        while done < total:
            with self._cv:
                while True:
                    if self._queue:
                        r, arr = self._queue[0]
                        est = self._est(r, min(r.m0, r.m_cap))
                        fits = (self._in_use + est <= self.budget and not self._blocked) or not self._running
                        if self._free_workers and fits:
                            self._queue.popleft()
                            w = self._free_workers.pop()
                            self._in_use += est
                            self._held[r.rid] = est
                            self._running.append(r.rid)
                            self.peak_bytes = max(self.peak_bytes, self._in_use)
                            self.peak_running = max(self.peak_running, len(self._running))
                            break
                    self._cv.wait(timeout=0.05)
            th = threading.Thread(target=self._run_one, args=(w, r, arr), daemon=True)
            th.start()
            threads.append(th)
            done += 1
        for th in threads:
            th.join()

    def serve(self, requests: list[Request]) -> list[Result]:
        """Run a request stream whose arrival_s are offsets from the start; returns results by rid."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        self._results = []
        self._t0 = time.perf_counter()
        disp = threading.Thread(target=self._dispatch, args=(len(reqs),), daemon=True)
        disp.start()
        for r in reqs:
            wait = r.arrival_s - self._now()
            if wait > 0:
                time.sleep(wait)
            with self._cv:
                self._queue.append((r, self._now()))
                self._cv.notify_all()
        disp.join()
        return sorted(self._results, key=lambda x: x.rid)


def summarize(results: list[Result], makespan_s: float | None = None) -> dict:
    lat = np.array([r.latency_s for r in results])
    span = makespan_s if makespan_s is not None else max(r.end_s for r in results) - min(r.arrival_s for r in results)
    return {"jobs": len(results), "jobs_per_s": len(results) / span if span > 0 else math.inf,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": span,
            "certified": int(sum(1 for r in results if r.status == P.OK))}


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> list[float]:
    """n arrival offsets of a Poisson process with the given rate (seeded)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n)).tolist()
