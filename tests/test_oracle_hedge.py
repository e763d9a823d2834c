"""Pins of the oracle's HEDGE-P rule (Sec. 6 progressive HEDGE; union bound of Sec. 2,
Eq. 1).

The SD bound eta_U comes from a two-sided Bernstein tail per set and a union bound over
the n^k sets of size <= k.  Checked here: both roots solve their defining equations, the
bound depends on (n, k) only through n^k, its large-m limit, the stopping rule against
HEDGE's sufficient condition SD <= eps C(S*)/2, that it covers the exact supremum
deviation on a graph small enough to enumerate every set, and a run's log.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

A = 1 - math.exp(-1)


@pytest.mark.parametrize("cov,m,n,k,i", [(0, 1000, 50, 3, 1), (400, 1000, 2000, 10, 2), (9000, 10**5, 10**6, 50, 5),
                                         (10**6, 10**6, 100, 100, 3)])
def test_roots_solve_their_equations(cov, m, n, k, i):
    stop, b = O.bounds_hedge(cov, m, n, k, 0.1, 0.05, i)
    L, nu, eta, C = b["LU"], b["nuU"], b["etaU"], b["C"]
    # the per-set deviation lam(v) solves m lam^2 = L (2 v + 2 lam / 3)
    v = min(nu, 0.25)
    assert m * eta * eta == pytest.approx(L * (2 * v + 2 * eta / 3), rel=1e-12)
    # nu_U is a fixed point of u = C / (1 - 1/e) + lam(u), and the larger one
    lam = lambda u: L / (3 * m) + math.sqrt((L / (3 * m)) ** 2 + 2 * u * L / m)
    assert nu == pytest.approx(C / A + lam(nu), rel=1e-12)
    assert nu * 1.001 > C / A + lam(nu * 1.001)
    # union bound over n^k sets, two tails, delta_i = delta / 2^i
    assert L == pytest.approx(math.log(2 * n**k * 2**i / 0.05), rel=1e-12)


def test_depends_on_n_and_k_only_through_n_to_the_k():
    for m, cov in ((5000, 1200), (10**6, 3 * 10**5)):
        _, b1 = O.bounds_hedge(cov, m, 100, 2, 0.1, 0.1, 3)
        _, b2 = O.bounds_hedge(cov, m, 10, 4, 0.1, 0.1, 3)
        _, b3 = O.bounds_hedge(cov, m, 10, 5, 0.1, 0.1, 3)
        assert b1["etaU"] == pytest.approx(b2["etaU"], rel=1e-12)
        assert b3["etaU"] > b2["etaU"]


def test_large_m_limit():
    # with C fixed, m eta_U^2 -> 2 min(C/(1-1/e), 1/4) L_U
    for C in (0.05, 0.4):
        m = 10**13
        _, b = O.bounds_hedge(int(C * m), m, 1000, 10, 0.1, 0.1, 1)
        assert m * b["etaU"] ** 2 == pytest.approx(2 * min(C / A, 0.25) * b["LU"], rel=1e-4)


def test_stop_rule_is_hedges_sufficient_condition():
    """Stop iff eta_U <= eps (C - eta_U)/2: C(S*) >= C - SD, so SD <= eta_U <= eps C(S*)/2."""
    m, n, k, eps = 10**6, 5000, 10, 0.2
    prev = False
    flips = 0
    for cov in range(0, m + 1, m // 200):
        stop, b = O.bounds_hedge(cov, m, n, k, eps, 0.1, 2)
        assert stop == (b["etaU"] <= eps * (b["C"] - b["etaU"]) / 2)
        flips += stop != prev
        prev = stop
    assert prev and flips == 1  # monotone in the coverage


def test_covers_exact_supremum_deviation_on_enumerable_graph():
    nx = pytest.importorskip("networkx")
    g = I.ba(10, 2, 4)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for v in range(g.n):
        for w in g.col[g.off[v]:g.off[v + 1]]:
            G.add_edge(v, int(w))
    paths = {(s, t): [set(p[1:-1]) for p in nx.all_shortest_paths(G, s, t)]
             for s in range(g.n) for t in range(g.n) if s != t}
    k = 2
    sets = [set(S) for r in range(1, k + 1) for S in itertools.combinations(range(g.n), r)]
    exact = [sum(sum(1 for p in ps if p & S) / len(ps) for ps in paths.values()) / (g.n * (g.n - 1)) for S in sets]
    og = O.Graph.of(g)
    m = 300
    worst = 0.0
    for seed in range(40):
        job = O.Job(og, 1000 + seed, 1)
        job.sample(m)
        h = job.hypergraph()
        mem = [set(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()) for j in range(m)]
        sd = max(abs(sum(1 for x in mem if x & S) / m - c) for S, c in zip(sets, exact))
        Sg, cov = job.greedy_cover(k)
        _, b = O.bounds_hedge(cov, m, g.n, k, 0.1, 0.1, 1)
        assert sd <= b["etaU"]
        worst = max(worst, sd / b["etaU"])
    assert worst > 0.05  # the bound is loose but not vacuous


def test_hedge_p_run_logs_and_needs_more_samples():
    g = O.Graph.of(I.ba(300, 3, 2))
    h = g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, m0=500, rule=1)
    c = g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, m0=500, rule=0)
    assert h["status"] == c["status"] == O.OK
    for i, row in enumerate(h["log"], start=1):
        stop, b = O.bounds_hedge(int(row[2]), int(row[1]), 300, 5, 0.2, 0.1, i)
        assert row[6] == b["C"] and row[9] == b["nuU"] and row[13] == b["etaU"] and bool(row[14]) == stop
        assert row[3] == row[4] == row[5] == row[7] == 0
    assert h["m_final"] >= c["m_final"]
    with pytest.raises(O.OracleError):
        g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, rule=2)
