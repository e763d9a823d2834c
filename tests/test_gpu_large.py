"""GPU parity on the high-diameter workloads at full size.

2048 x 2048 grid with 1% of edges rewired (n = 4,194,304; d(s,t) around 30-40,
so waves run dozens of levels), and directed R-MAT scale 22 (67M arc draws; the
in-arc CSR is built on the GPU; many targets unreachable).  The oracle computes
sampled hyper-edges one by one; every hyper-edge must also be the interior of
a path whose consecutive nodes are joined by arcs.
"""
import numpy as np
import pytest

import oracle as O
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
    og = O.Graph.of(g)
    for j in picks:
        rc, s, tt, d, path = og.hyperedge(seed, j)
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
    return h


def test_grid2048_rewired_sampled_parity():
    g = I.grid_rewired(2048, 2048, 0.01, seed=1)
    h = check_sampled(g, seed=1, m=600, picks=[0, 1, 255, 256, 511, 599])
    assert h["d"].min() >= 1 and h["d"].max() > 20


def test_rmat22_directed_sampled_parity():
    g = I.rmat(22, 16, seed=1, directed=True, keep_lcc=False)
    h = check_sampled(g, seed=1, m=2100, picks=[0, 3, 2047, 2048, 2099])
    assert (h["d"] == -1).any() and (h["d"] >= 2).any()
