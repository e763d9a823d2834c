"""GPU parity of a whole round at the benchmark's sizes, element by element.

R-MAT scale 18 LCC (n = 174,078): every one of 8,192 hyper-edges, greedyCover at
k = 50 and 100 (picks and coverage), the full R matrix, every Rnum, Wnum, b and the
FP64 bounds, against the oracle's own store of the same 8,192 samples (drawn by index
range in spawned worker processes and merged; samples are functions of their index).
At this size the select runs many blocks per row (multi-block histogram merge) and the
cooperative greedy contends across all SMs.  The same store is checked with the
bidirectional sampler forced through its other paths: the smallest node table (many
searches move to the large table), no small table, a short queue (searches handed
to the bit-parallel sampler), and whole-CTA searches only, with and without the
smallest node table.  Epoch wrap: a few CTAs draw more than
65,535 searches per search group on a small graph, so the 16-bit epochs of the node
tables wrap and the tables are cleared.
"""
import math

import os

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
    assert job.sampler_info()["escalated"] == 0  # by default a hub-heavy graph starts with whole-CTA searches
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
        # and greedyCover as an 8-CTA cluster and in the cooperative grid form (graphs over
        # 921,600 nodes use it)
        for var, val in (("CEN_GREEDY_CLUSTER", "8"), ("CEN_GREEDY_GRID", "1")):
            os.environ[var] = val
            try:
                S3, cov3 = job.greedy_cover(k)
            finally:
                del os.environ[var]
            assert S3.tolist() == oS.tolist() and cov3 == ocov, var
        for i in (1, 4):
            st, bd = P.bounds(cov, M18, int(Rnum.sum()), wl.t, Wnum, b, wl.eps, wl.delta, i)
            ost, obd = O.bounds(ocov, M18, int(oRnum.sum()), wl.t, oWnum, ob, wl.eps, wl.delta, i)
            assert st == ost and bd == obd
    assert len(S) == 100 and cov > 0


@pytest.mark.parametrize("table,queue,warps", [(1024, 0, 1), (0, 0, 1), (0, 2048, 1), (-1, 0, 0), (1024, 0, 0)])
def test_rmat18_store_through_every_sampler_path(rmat18, table, queue, warps):
    wl, _, ref = rmat18
    job = P.Job(P.Graph.of(wl.graph), wl.seed, wl.t)
    job.tune(bidir_table=table, bidir_queue=queue or None, bidir_warps=warps)
    job.sample(M18)
    store_equal(job.samples(), ref)
    info = job.sampler_info()
    assert (info["escalated"] > 0) == (warps != 0)  # warp searches that outgrew a warp went to a CTA
    if table == 1024:
        assert info["migrated"] > 0  # searches that filled half of the small table moved to the large one
    if queue:
        assert info["deferred_search"] > 0  # balls beyond the queue went to the bit-parallel sampler


@pytest.mark.parametrize("table,warps,m", [(0, 0, 450_000), (1024, 0, 450_000), (1024, 1, 1_400_000)])
def test_epoch_wrap_of_the_node_tables(table, warps, m):
    """A 1 MiB workspace budget leaves four or five CTAs, whose search groups draw more
    than 65,535 searches each, so their 16-bit table epochs wrap and the tables are
    cleared: whole-CTA searches in the large table only (table 0) or in the small table
    (table 1024), and warp searches in the warps' own tables (four groups per CTA)."""
    g = I.ba(2000, 4, 1)
    job = P.Job(P.Graph.of(g), 3, 4)
    job.tune(bidir_budget=1 << 20, bidir_queue=2000, bidir_table=table, bidir_warps=warps)
    job.sample(m)
    info = job.sampler_info()
    groups = info["slots"] * (4 if warps else 1)
    assert 1 <= info["slots"] <= 5 and m / groups > 1.1 * 65535, info
    assert info["deferred_search"] == 0
    with shards.Pool(g) as pool:
        ref = pool.job(3, 4, m).hypergraph()
    store_equal(job.samples(), ref)
