"""GPU parity of a whole round at the benchmark's sizes, element by element.

R-MAT scale 18 LCC (n = 174,078): every one of 8,192 hyper-edges, greedyCover at
k = 50 and 100 (picks and coverage), the full R matrix, every Rnum, Wnum, b and the
FP64 bounds, against the oracle's own store of the same 8,192 samples (drawn by index
range in spawned worker processes and merged; samples are functions of their index).
At this size the select runs many blocks per row (multi-block histogram merge) and the
cooperative greedy contends across all SMs.  The same store is checked with the
bidirectional sampler forced through its other paths: the smallest node table (many
searches move to the large table), no small table, and a short queue (searches handed
to the bit-parallel sampler).  Epoch wrap: five CTAs draw 90,000 searches each on a
small graph, so the 16-bit epochs of both node tables wrap and the tables are cleared.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import shards
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")

M18 = 8192


@pytest.fixture(scope="module")
def rmat18():
    wl = I.rmat18_lcc()
    with shards.Pool(wl.graph) as pool:
        ojob = pool.job(wl.seed, wl.t, M18)
    return wl, ojob, ojob.hypergraph()


def store_equal(h, ref):
    for key in ("hoff", "s", "t", "d"):
        assert np.array_equal(h[key], ref[key]), key
    members = int(ref["hoff"][-1])
    assert np.array_equal(h["hmem"][:members], ref["hmem"][:members])


def test_rmat18_whole_round_against_the_oracle(rmat18):
    wl, ojob, ref = rmat18
    g = wl.graph
    job = P.Job(P.Graph.of(g), wl.seed, wl.t)
    job.sample(M18)
    store_equal(job.samples(), ref)
    oR, oc = ojob.rade_matrix()
    for k in (50, 100):
        S, cov, Rnum, Wnum, b = job.cover_and_mcera(k)
        oS, ocov = ojob.greedy_cover(k)
        oRnum, oWnum, ob = ojob.mcera(k)
        assert S.tolist() == oS.tolist() and cov == ocov, k
        assert np.array_equal(Rnum, oRnum) and Wnum == oWnum and b == ob, k
        R, c = job.rade()
        assert np.array_equal(R, oR.T) and np.array_equal(c, oc)
        # the same through the separate calls
        S2, cov2 = job.greedy_cover(k)
        R2, W2, b2 = job.mcera(k)
        assert S2.tolist() == oS.tolist() and cov2 == ocov and np.array_equal(R2, oRnum) and W2 == oWnum
        for i in (1, 4):
            st, bd = P.bounds(cov, M18, int(Rnum.sum()), wl.t, Wnum, b, wl.eps, wl.delta, i)
            ost, obd = O.bounds(ocov, M18, int(oRnum.sum()), wl.t, oWnum, ob, wl.eps, wl.delta, i)
            assert st == ost and bd == obd
    assert len(S) == 100 and cov > 0


@pytest.mark.parametrize("table,queue", [(1024, 0), (0, 0), (0, 2048)])
def test_rmat18_store_through_every_sampler_path(rmat18, table, queue):
    wl, _, ref = rmat18
    job = P.Job(P.Graph.of(wl.graph), wl.seed, wl.t)
    job.tune(bidir_table=table, bidir_queue=queue or None)
    job.sample(M18)
    store_equal(job.samples(), ref)
    info = job.sampler_info()
    if table == 1024:
        assert info["migrated"] > 0  # searches that filled half of the small table moved to the large one
    if queue:
        assert info["deferred_search"] > 0  # balls beyond the queue went to the bit-parallel sampler


@pytest.mark.parametrize("table", [0, 1024])
def test_epoch_wrap_of_the_node_tables(table):
    """Five CTAs (a 1 MiB workspace budget) draw 450,000 searches between them, so each
    passes 65,535 searches and its table epoch wraps (table 0: the large table's epoch
    advances per search; table 1024: the small table's)."""
    g = I.ba(2000, 4, 1)
    m = 450_000
    job = P.Job(P.Graph.of(g), 3, 4)
    job.tune(bidir_budget=1 << 20, bidir_queue=2000, bidir_table=table)
    job.sample(m)
    info = job.sampler_info()
    assert 1 <= info["slots"] <= 5 and m / info["slots"] > 1.3 * 65535
    assert info["deferred_search"] == 0
    with shards.Pool(g) as pool:
        ref = pool.job(3, 4, m).hypergraph()
    store_equal(job.samples(), ref)
