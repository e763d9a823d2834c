"""Degenerate inputs through the C ABI, against the oracle: a job with no samples, graphs of
two nodes (every pair adjacent, or none reachable), k beyond n, and t at its bounds."""
import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2306_03651_gb300")


def two_nodes(edge: bool):
    if edge:
        return I.from_edges(2, [0], [1], False)
    return I.Graph(2, np.zeros(3, np.int64), np.zeros(0, np.int32), False, "two isolated nodes")


def test_job_without_samples():
    g = I.ba(200, 2, 3)
    job = P.Job(P.Graph.of(g), 1, 5)
    job.sample(0)
    assert job.size() == (0, 0)
    S, cov = job.greedy_cover(4)
    assert len(S) == 0 and cov == 0
    Rn, Wn, b = job.mcera(4)
    assert not Rn.any() and Wn == 0 and b == 0
    S, cov, Rn, Wn, b = job.cover_and_mcera(4)
    assert len(S) == 0 and cov == 0 and not Rn.any() and Wn == 0 and b == 0


@pytest.mark.parametrize("edge", [True, False])
def test_two_node_graphs_give_empty_hyperedges(edge):
    g = two_nodes(edge)
    job = P.Job(P.Graph.of(g), 7, 3)
    job.sample(500)
    oj = O.Job(O.Graph.of(g), 7, 3)
    oj.sample(500)
    a, b = job.samples(), oj.hypergraph()
    for key in ("hoff", "s", "t", "d", "hmem"):
        assert np.array_equal(a[key], b[key]), key
    assert a["hoff"][-1] == 0 and (a["d"] == (1 if edge else -1)).all()
    S, cov, Rn, Wn, bh = job.cover_and_mcera(2)
    assert len(S) == 0 and cov == 0 and not Rn.any() and Wn == 0 and bh == 0
    r = P.run(P.Graph.of(g), 1, 0.1, 0.1, 3, 7, m0=100, m_cap=1000)
    assert r["status"] == P.ENOTCERTIFIED


@pytest.mark.parametrize("t", [1, 4096])
def test_t_at_its_bounds_and_k_beyond_n(t):
    g = I.ba(60, 2, 5)
    job = P.Job(P.Graph.of(g), 3, t)
    job.sample(700)
    oj = O.Job(O.Graph.of(g), 3, t)
    oj.sample(700)
    k = 80  # more than n: the greedy stops once no node adds coverage
    S, cov, Rn, Wn, b = job.cover_and_mcera(k)
    S2, cov2 = oj.greedy_cover(k)
    Rn2, Wn2, b2 = oj.mcera(k)
    assert S.tolist() == S2.tolist() and cov == cov2 and len(S) < g.n
    assert np.array_equal(Rn, Rn2) and Wn == Wn2 and b == b2
