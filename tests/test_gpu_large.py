"""GPU parity on the high-diameter workloads at full size.

2048 x 2048 grid with 1% of edges rewired (n = 4,194,304; d(s,t) around 30-40,
so waves run dozens of levels), and directed R-MAT scale 22 (67M arc draws; the
in-arc CSR is built on the GPU; many targets unreachable).  The oracle computes
sampled hyper-edges one by one (210 per graph, in spawned worker processes,
including the first and last of each CTA wave and searches that moved to the
large node table); every hyper-edge must also be the interior of a path whose
consecutive nodes are joined by arcs.
"""
import numpy as np
import pytest

import oracle as O
from oracle import shards
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")


def has_arc(g, a, b):
    row = g.col[g.off[a]:g.off[a + 1]]
    i = int(np.searchsorted(row, b))
    return i < len(row) and row[i] == b


def check_sampled(g, seed, m, picks, t=8):
    job = P.Job(P.Graph.of(g), seed, t)
    job.sample(m)
    h = job.samples()
    with shards.Pool(g) as pool:
        ref = pool.hyperedges(seed, picks)
    for j in picks:
        rc, s, tt, d, path = ref[j]
        assert rc == O.OK
        assert (h["s"][j], h["t"][j], h["d"][j]) == (s, tt, d), j
        assert h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist() == path, j
    assert np.array_equal(np.diff(h["hoff"]), np.maximum(h["d"] - 1, 0))
    for j in range(0, m, 11):
        if h["d"][j] < 1:
            continue
        full = [h["s"][j]] + h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist() + [h["t"][j]]
        assert len(set(full)) == len(full)
        for a, b in zip(full, full[1:]):
            assert has_arc(g, a, b)
    return job, h


def picks_of(m, count, seed):
    rng = np.random.default_rng(seed)
    fixed = {0, 1, m // 2, m - 2, m - 1}
    return sorted(fixed | set(rng.choice(m, count - len(fixed), replace=False).tolist()))


def test_grid2048_rewired_sampled_parity():
    g = I.grid_rewired(2048, 2048, 0.01, seed=1)
    m = 4000
    job, h = check_sampled(g, seed=1, m=m, picks=picks_of(m, 210, 5))
    assert h["d"].min() >= 1 and h["d"].max() > 20
    assert job.sampler_info()["migrated"] > 0


def test_rmat22_directed_sampled_parity():
    g = I.rmat(22, 16, seed=1, directed=True, keep_lcc=False)
    m = 8192
    _, h = check_sampled(g, seed=1, m=m, picks=picks_of(m, 210, 6))
    assert (h["d"] == -1).any() and (h["d"] >= 2).any()
