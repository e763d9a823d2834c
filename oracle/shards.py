"""The oracle over several host processes -- TEST INFRASTRUCTURE ONLY.

A sample is a function of (graph, seed, sample index) alone (Sec. 5 sampleHEs with
Philox keyed by the index), so index ranges can be drawn in separate processes and
stored into one oracle job in index order (`Job.append`); the result equals a single
job's samples.  Greedy, AMCERA and bounds then run on that job as usual.  Workers are
spawned (never forked), so a pool may start after the parent has used CUDA, and each
worker memory-maps the graph from a temporary directory instead of receiving it
through a pipe.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

_G = None  # the worker's oracle graph


def _init(path: str, n: int, directed: bool):
    global _G
    import oracle as O
    off = np.load(os.path.join(path, "off.npy"), mmap_mode="r")
    col = np.load(os.path.join(path, "col.npy"), mmap_mode="r")
    _G = O.Graph(n, np.ascontiguousarray(off), np.ascontiguousarray(col), directed)


def _range(args):
    import oracle as O
    seed, t, a, b = args
    job = O.Job(_G, seed, t)
    job.sample_from(a, b - a)
    h = job.hypergraph()
    members = int(h["hoff"][-1])
    return a, {"hoff": h["hoff"], "hmem": h["hmem"][:members], "s": h["s"][: b - a], "t": h["t"][: b - a],
               "d": h["d"][: b - a]}


def _one(args):
    seed, j = args
    return j, _G.hyperedge(seed, j)


class Pool:
    """Spawned oracle workers that share one graph (`with Pool(g, procs) as p:`)."""

    def __init__(self, g, procs: int | None = None):
        self.g = g
        self.procs = procs or max(1, min(16, os.cpu_count() or 1))
        self._dir = tempfile.TemporaryDirectory(prefix="oracle_shards_")
        np.save(os.path.join(self._dir.name, "off.npy"), np.ascontiguousarray(g.off, np.int64))
        np.save(os.path.join(self._dir.name, "col.npy"), np.ascontiguousarray(g.col, np.int32))
        self._pool = mp.get_context("spawn").Pool(self.procs, initializer=_init,
                                                  initargs=(self._dir.name, int(g.n), bool(g.directed)))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
            self._dir.cleanup()

    def job(self, seed: int, t: int, m: int, chunk: int | None = None):
        """An oracle Job holding samples 0 .. m-1, drawn in index ranges by the workers."""
        import oracle as O
        chunk = chunk or max(1, -(-m // (4 * self.procs)))
        tasks = [(seed, t, a, min(m, a + chunk)) for a in range(0, m, chunk)]
        parts = dict(self._pool.map(_range, tasks))
        job = O.Job(O.Graph.of(self.g), seed, t)
        for a in sorted(parts):
            job.append(a, parts[a])
        assert job.m == m
        return job

    def hyperedges(self, seed: int, ids):
        """{j: (rc, s, t, d, path)} of the oracle's hyper-edge j, one by one."""
        return dict(self._pool.map(_one, [(seed, int(j)) for j in ids]))
