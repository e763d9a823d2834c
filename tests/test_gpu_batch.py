"""Batched Algorithm 1 (cen_run_batch): every job's result equals cen_run on
the same spec alone, whatever the number of workers and the order jobs finish in."""
import numpy as np
import pytest

from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")


def specs():
    out = []
    for j, (n, d, k) in enumerate([(300, 2, 5), (2000, 4, 10), (800, 3, 20), (1500, 5, 8), (400, 2, 3), (3000, 6, 15)]):
        g = P.Graph.of(I.ba(n, d, 100 + j))
        out.append(dict(graph=g, k=k, eps=0.15, delta=0.1, t=8, seed=j, m0=500))
    return out


def same(a, b):
    assert a["status"] == b["status"] and a["S"].tolist() == b["S"].tolist()
    assert a["covered"] == b["covered"] and a["m_final"] == b["m_final"] and a["rounds"] == b["rounds"]
    assert np.array_equal(a["log"], b["log"])


def test_batch_equals_individual_runs():
    jobs = specs()
    alone = [P.run(j["graph"], j["k"], j["eps"], j["delta"], j["t"], j["seed"], m0=j["m0"]) for j in jobs]
    for workers in (1, 3, 8):
        res = P.run_batch(jobs, nworkers=workers)
        for a, r in zip(alone, res):
            same(a, r)
            assert r["end_s"] >= r["start_s"] >= 0


def test_batch_rejects_bad_arguments():
    with pytest.raises(P.CenError):
        P.run_batch([], nworkers=0)


def test_run_result_struct_equals_run():
    for j in specs()[:3]:
        r = P.run_result(j)
        a = P.run(j["graph"], j["k"], j["eps"], j["delta"], j["t"], j["seed"], m0=j["m0"])
        same(a, r)
        assert r["status"] == a["status"] and r["seconds"] > 0
