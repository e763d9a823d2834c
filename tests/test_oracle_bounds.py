"""Pins of the oracle's FP64 bounds (Thm. 4.4, Eq. 2), the stopping
test of Algorithm 1, and the progressive loop.

Special cases with closed forms (C = 0, w = 0, R~ = 0), the equivalence of the
stopping line with the inequality chain in the proof of Prop. 4.5, the
monotonicity of eta, its large-m limit 2 A, and the schedule
(delta_i = delta / 2^i, m_i = m0 2^(i-1)), and Sec. 4.2's schedule (its guess
solves the no-deviation eta for m; growth by alpha).  End to end: on a graph small enough
for exact set betweenness, the certified set reaches (1 - 1/e - eps) of the
brute-force optimum.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

A = 1 - math.exp(-1)


def L_of(delta, i):
    return math.log(5 * 2**i / delta)


@pytest.mark.parametrize("m,i", [(1000, 1), (64000, 7), (10**6, 3)])
def test_zero_coverage_closed_forms(m, i):
    # C = 0: xi = nu = 2 L/m.  A = 0, w = 0: Rt = 0, R = 2 L/m,
    # eta = 4 L/m + sqrt(2 L (2L/m + 8L/m) / m) + L/(3m) = (4 + sqrt(20) + 1/3) L/m
    stop, b = O.bounds(0, m, 0, 10, 0, 0, 0.1, 0.1, i)
    L = L_of(0.1, i)
    assert b["C"] == 0 and b["A"] == 0 and b["w"] == 0
    assert b["xi"] == pytest.approx(2 * L / m, rel=1e-14)
    assert b["nu"] == pytest.approx(2 * L / m, rel=1e-14)
    assert b["Rt"] == 0
    assert b["R"] == pytest.approx(2 * L / m, rel=1e-14)
    assert b["eta"] == pytest.approx((4 + math.sqrt(20) + 1 / 3) * L / m, rel=1e-14)
    assert not stop  # C = 0 can never be certified


def test_no_variance_keeps_amcera():
    stop, b = O.bounds(500, 1000, 1234, 10, 0, 0, 0.1, 0.1, 2)
    assert b["Rt"] == b["A"] == pytest.approx(1234 / (10 * 1000), rel=1e-15)
    assert b["C"] == 0.5


def test_scaled_inputs():
    # every bound depends on the sample through C, A, w and m only
    s1, b1 = O.bounds(300, 1000, 200, 10, 900, 3, 0.05, 0.1, 2)
    s2, b2 = O.bounds(600, 2000, 400, 10, 1800, 3, 0.05, 0.1, 2)
    for key in ("C", "A", "w"):
        assert b1[key] == pytest.approx(b2[key], rel=1e-15)
    assert b2["eta"] < b1["eta"] and b2["xi"] < b1["xi"]


def test_stop_equals_prop_main_chain():
    """Alg. 1's test a((a-eps) xi + eta) <= eps C is the middle inequality of the proof of
    Prop. 4.5: C/a + xi <= (C - eta)/(a - eps)."""
    rng = np.random.default_rng(0)
    agree = 0
    for _ in range(3000):
        m = int(rng.integers(1000, 10**7))
        cov = int(rng.integers(0, m + 1))
        t = int(rng.integers(1, 100))
        Rsum = int(rng.integers(0, 5 * t * math.isqrt(m) + 1))
        Wnum = int(rng.integers(0, 4 * m + 1))
        b = int(rng.integers(0, 20))
        eps = float(rng.uniform(0.001, 0.5))
        i = int(rng.integers(1, 12))
        stop, v = O.bounds(cov, m, Rsum, t, Wnum, b, eps, 0.1, i)
        lhs = v["C"] / A + v["xi"]
        rhs = (v["C"] - v["eta"]) / (A - eps)
        if abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs)):
            continue  # rounding decides at the boundary
        assert stop == (lhs <= rhs)
        agree += stop
    assert agree > 0


def test_eta_monotone_and_limit():
    base = dict(covered=4000, m=10000, Rsum=300, t=10, Wnum=20000, b=4, eps=0.05, delta=0.1, i=3)
    def eta(**kw):
        a = dict(base, **kw)
        return O.bounds(a["covered"], a["m"], a["Rsum"], a["t"], a["Wnum"], a["b"], a["eps"], a["delta"], a["i"])[1]
    e0 = eta()["eta"]
    assert eta(Rsum=600)["eta"] > e0
    assert eta(Wnum=40000)["eta"] > e0
    assert eta(b=8)["eta"] > e0
    assert eta(i=4)["eta"] > e0  # smaller delta_i
    # fixed C, A, w: eta -> 2 A as m grows (numerators scaled with m)
    for m in (10**6, 10**8, 10**10):
        s = m // 10000
        v = eta(covered=4000 * s, m=m, Rsum=300 * s, Wnum=20000 * s)
        assert v["A"] == pytest.approx(0.003)
    assert v["eta"] == pytest.approx(2 * 0.003, rel=0.05)


def test_run_schedule_and_first_stop():
    g = O.Graph.of(I.ba(300, 3, 2))
    r = g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, m0=500)
    assert r["status"] == O.OK
    log = r["log"]
    for row_i, row in enumerate(log, start=1):
        assert row[0] == row_i and row[1] == 500 * 2 ** (row_i - 1)
        stop, b = O.bounds(int(row[2]), int(row[1]), int(row[3]), 10, int(row[4]), int(row[5]), 0.2, 0.1, row_i)
        assert stop == bool(row[14])
        assert b["eta"] == row[13] and b["xi"] == row[10]
    assert all(row[14] == 0 for row in log[:-1]) and log[-1][14] == 1
    assert r["m_final"] == log[-1][1] and r["covered"] == log[-1][2]


def test_run_not_certified_on_empty_hyperedges():
    # complete graph: every hyper-edge is empty, C = 0 forever
    n = 8
    e = np.array([(a, b) for a in range(n) for b in range(a + 1, n)], np.int32)
    g = O.Graph.of(I.from_edges(n, e[:, 0], e[:, 1], False))
    r = g.run(k=2, eps=0.1, delta=0.1, t=4, seed=1, m0=100, m_cap=1600)
    assert r["status"] == O.ENOTCERTIFIED and r["m_final"] == 1600 and r["covered"] == 0
    assert len(r["S"]) == 0


def test_run_rejects_bad_arguments():
    g = O.Graph.of(I.ba(30, 2, 1))
    for kw in (dict(k=0), dict(eps=0.0), dict(eps=0.7), dict(delta=1.0), dict(t=0)):
        args = dict(k=3, eps=0.1, delta=0.1, t=4, seed=1)
        args.update(kw)
        with pytest.raises(O.OracleError):
            g.run(**args)


def test_certified_set_is_within_guarantee_on_tiny_graph():
    """Prop. 4.5: C(S) >= (1 - 1/e - eps) C(S*), checked with exact set betweenness."""
    nx = pytest.importorskip("networkx")
    g = I.ba(14, 2, 6)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for v in range(g.n):
        for w in g.col[g.off[v]:g.off[v + 1]]:
            G.add_edge(v, int(w))
    pairs = {}
    for s in range(g.n):
        for t in range(g.n):
            if s != t:
                pairs[(s, t)] = [set(p[1:-1]) for p in nx.all_shortest_paths(G, s, t)]
    def B(S):
        S = set(S)
        return sum(sum(1 for p in ps if p & S) / len(ps) for ps in pairs.values()) / (g.n * (g.n - 1))
    k, eps = 2, 0.3
    opt = max(B(S) for S in itertools.combinations(range(g.n), k))
    og = O.Graph.of(g)
    for seed in range(3):
        r = og.run(k=k, eps=eps, delta=0.1, t=10, seed=seed, m0=1000)
        assert r["status"] == O.OK
        assert B(r["S"]) >= (1 - 1 / math.e - eps) * opt


@pytest.mark.parametrize("C,eps,i", [(1.0, 0.05, 1), (0.4, 0.01, 3), (0.05, 0.2, 7)])
def test_schedule_guess_solves_the_optimistic_bound(C, eps, i):
    """Sec. 4.2: with R = 0 and nu = 1, eta(m) = sqrt(2 L/m) + L/(3 m) equals the
    target eps C / (1 - 1/e) at the guess, and is above it for smaller m."""
    m = O.schedule_guess(C, eps, 0.1, i)
    L = L_of(0.1, i)
    eta = lambda mm: math.sqrt(2 * L / mm) + L / (3 * mm)
    assert eta(m) == pytest.approx(eps * C / A, rel=1e-12)
    assert eta(0.99 * m) > eps * C / A > eta(1.01 * m)
    assert O.schedule_guess(0.0, eps, 0.1, i) == 0.0


def test_paper_schedule_grows_geometrically_and_follows_the_guess():
    g = O.Graph.of(I.ba(300, 3, 2))
    r = g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, m0=500, schedule=1, alpha=1.2)
    assert r["status"] == O.OK
    ms = [int(row[1]) for row in r["log"]]
    assert ms[0] == max(500, math.ceil(O.schedule_guess(1.0, 0.2, 0.1, 1)))
    for prev, cur, row, i in zip(ms, ms[1:], r["log"], range(2, 99)):
        assert cur >= math.ceil(1.2 * prev) and cur > prev
        assert cur == max(math.ceil(1.2 * prev), math.ceil(O.schedule_guess(row[6], 0.2, 0.1, i)))
    # the doubling schedule is unchanged
    d = g.run(k=5, eps=0.2, delta=0.1, t=10, seed=3, m0=500)
    assert [int(row[1]) for row in d["log"]] == [500 * 2 ** q for q in range(len(d["log"]))]


@pytest.mark.parametrize("rule", [0, 1])
def test_predicting_schedule_targets_the_next_stopping_test(rule):
    """Schedule 2: the next size is the smallest at which the next round's stopping test
    passes when C and w hold and the AMCERA shrinks as 1/sqrt(m); checked by re-evaluating
    the oracle's own bounds just above and just below the predicted size, with the sums scaled."""
    g = O.Graph.of(I.rmat(10, 8, seed=2))
    eps, delta, k, t = 0.1, 0.1, 8, 20
    r = g.run(k=k, eps=eps, delta=delta, t=t, seed=4, m0=1000, schedule=2, alpha=1.2, rule=rule)
    p = g.run(k=k, eps=eps, delta=delta, t=t, seed=4, m0=1000, schedule=1, alpha=1.2, rule=rule)
    assert r["status"] == p["status"] == O.OK
    assert len(r["log"]) < len(p["log"])
    ms = [int(row[1]) for row in r["log"]]

    def passes(row, mp, i):
        m, C = row[1], row[6]
        if rule == 1:
            return O.bounds_hedge(round(C * mp), mp, g.n, k, eps, delta, i)[0]
        # integer sums whose fractions are C, A sqrt(m/mp), w at size mp (b = 1 carries w)
        Rsum = round(row[7] * math.sqrt(m / mp) * t * mp)
        return O.bounds(round(C * mp), mp, Rsum, t, round(row[8] * mp), 1, eps, delta, i)[0]

    predicted = 0
    for i, (row, nxt) in enumerate(zip(r["log"], ms[1:]), start=1):
        floor = max(math.ceil(1.2 * row[1]), math.ceil(O.schedule_guess(row[6], eps, delta, i + 1)))
        predicted += nxt > floor
        if nxt > floor:  # the prediction decided: it passes there and not earlier (rounding the sums aside)
            assert passes(row, math.ceil(nxt * 1.001), i + 1) and not passes(row, math.floor(nxt * 0.999), i + 1)
    assert predicted >= 1 and all(b > a for a, b in zip(ms, ms[1:]))
