"""Serving loop: requests admitted mid-flight by HBM budget and run
concurrently give exactly the results they give alone."""
import numpy as np
import pytest

from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")


def setup():
    from paper_2306_03651_gb300 import serve as S
    graphs = {f"ba{j}": P.Graph.of(I.ba(n, d, 50 + j)) for j, (n, d) in enumerate([(500, 2), (1500, 4), (3000, 3)])}
    reqs = []
    rng = np.random.default_rng(1)
    arr = S.poisson_arrivals(10, 40.0, seed=2)
    for i in range(10):
        reqs.append(S.Request(rid=i, graph=f"ba{i % 3}", k=int(rng.integers(3, 20)), eps=float(rng.choice([0.1, 0.2])),
                              delta=0.1, t=8, seed=100 + i, arrival_s=arr[i], m0=500, m_cap=1 << 22))
    return S, graphs, reqs


@pytest.mark.parametrize("workers,budget", [(4, None), (3, 1)])
def test_served_results_equal_alone(workers, budget):
    S, graphs, reqs = setup()
    srv = S.Server(graphs, workers=workers, hbm_budget_bytes=budget)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(10))
    for q, r in zip(reqs, res):
        alone = P.run(graphs[q.graph], q.k, q.eps, q.delta, q.t, q.seed, m0=q.m0, m_cap=q.m_cap)
        assert r.status == alone["status"] == P.OK
        assert r.S.tolist() == alone["S"].tolist() and r.covered == alone["covered"]
        assert r.m_final == alone["m_final"] and np.array_equal(r.log, alone["log"])
        assert r.end_s >= r.start_s >= r.arrival_s - 1e-6
    if budget == 1:
        assert srv.peak_running == 1  # a 1-byte budget admits one job at a time
    summ = S.summarize(res)
    assert summ["jobs"] == 10 and summ["certified"] == 10 and summ["p99_latency_s"] >= summ["p50_latency_s"]
