"""Autotuner for the sampler's launch parameters.

The sampler choice (bidirectional with the bit-parallel fallback, or
bit-parallel waves only), the bidirectional sampler's node-table size and
search granularity (warps, or whole CTAs), and
the wave parameters (wave width, wave pipelines in flight, top-down/bottom-up
switch) only change speed and memory: every configuration yields the same
samples.  ``autotune`` times one probe round per
configuration on the caller's graph (after an untimed call that sizes that
configuration's workspace), checks that all configurations produced
identical hyper-edges, and stores the fastest as the graph's default
(``cen_graph_set_param``) so that later jobs, ``run``, ``run_batch`` and the
serving loop use it.
"""
from __future__ import annotations

import hashlib
import itertools
import time

import numpy as np

from . import cen as P

DEFAULT_GRID = dict(sampler=(0, 1), bidir_table=(-1, 0, 8192), wave_streams=(1, 4))
PARAM_IDS = {"wave_words": P.PARAM_WAVE_WORDS, "wave_streams": P.PARAM_WAVE_STREAMS, "push_ratio": P.PARAM_PUSH_RATIO,
             "level_budget": P.PARAM_LEVEL_BUDGET, "sampler": P.PARAM_SAMPLER, "bidir_budget": P.PARAM_BIDIR_BUDGET,
             "bidir_queue": P.PARAM_BIDIR_QUEUE, "bidir_table": P.PARAM_BIDIR_TABLE, "bidir_warps": P.PARAM_BIDIR_WARPS}
# the bidirectional sampler's own choices, for tuning many graphs (the batched form)
SAMPLER_GRID = dict(bidir_warps=(0, 1), bidir_table=(-1, 0))


def _digest(h: dict) -> str:
    m = hashlib.sha256()
    for key in ("hoff", "hmem", "s", "t", "d"):
        m.update(np.ascontiguousarray(h[key]).tobytes())
    return m.hexdigest()


def autotune(graph: "P.Graph", t: int = 10, probe_pairs: int = 8192, seed: int = 987654321, grid: dict | None = None,
             apply: bool = True) -> dict:
    """Returns dict(best=config, seconds=..., table=[(config, seconds)], digest=...)."""
    import torch
    grid = grid or DEFAULT_GRID
    keys = sorted(grid)
    table, digests = [], set()
    for combo in itertools.product(*(grid[k] for k in keys)):
        cfg = dict(zip(keys, combo))
        warm = P.Job(graph, seed + 1, t)  # untimed: sizes this configuration's workspace (kept for reuse)
        warm.tune(**cfg)
        warm.sample(min(probe_pairs, 2048))
        warm.close()
        job = P.Job(graph, seed, t)
        job.tune(**cfg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        job.sample(probe_pairs)
        torch.cuda.synchronize()
        table.append((cfg, time.perf_counter() - t0))
        digests.add(_digest(job.samples()))
        job.close()
    if len(digests) != 1:
        raise RuntimeError("autotune: configurations disagree on the samples")
    best, secs = min(table, key=lambda x: x[1])
    if apply:
        for name, value in best.items():
            graph.set_param(PARAM_IDS[name], value)
    return dict(best=best, seconds=secs, table=table, digest=digests.pop())
