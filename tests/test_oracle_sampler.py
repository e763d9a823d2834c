"""Pins of the oracle's hyper-edge sampler (Sec. 3.1 set betweenness; Sec. 5 sampleHEs).

sigma-BFS against networkx's shortest-path enumeration and grid closed forms,
the overflow boundary at 2^128, degenerate graphs (star, complete, tree,
unreachable), a chi-square test of (s, t, path) frequencies against the exact
probabilities 1 / (n (n-1) sigma_st), and the sample estimate against exact
set betweenness by all-pairs enumeration.
"""
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2306_03651_gb300 import inputs as I

nx = pytest.importorskip("networkx")


def nx_to_graph(G, directed=None):
    directed = G.is_directed() if directed is None else directed
    G = nx.convert_node_labels_to_integers(G, ordering="sorted")
    e = np.array(list(G.edges()), dtype=np.int32).reshape(-1, 2)
    return I.from_edges(G.number_of_nodes(), e[:, 0], e[:, 1], directed)


def graph_to_nx(g):
    G = nx.DiGraph() if g.directed else nx.Graph()
    G.add_nodes_from(range(g.n))
    for v in range(g.n):
        for w in g.col[g.off[v]:g.off[v + 1]]:
            G.add_edge(v, int(w))
    return G


def small_graphs():
    return {
        "ba30": I.ba(30, 2, 3),
        "petersen": nx_to_graph(nx.petersen_graph()),
        "cycle8": nx_to_graph(nx.cycle_graph(8)),
        "grid5x4": I.grid_rewired(5, 4, 0.0, 1),
        "digraph": nx_to_graph(nx.gnp_random_graph(25, 0.12, seed=4, directed=True)),
        "rewired": I.grid_rewired(6, 6, 0.2, 9),
    }


@pytest.mark.parametrize("name", list(small_graphs()))
def test_sigma_bfs_matches_networkx(name):
    g = small_graphs()[name]
    G = graph_to_nx(g)
    og = O.Graph.of(g)
    rng = np.random.default_rng(1)
    for _ in range(12):
        s, t = (int(x) for x in rng.choice(g.n, 2, replace=False))
        d, dist, sig, ovf = og.sigma_bfs(s, t)
        lengths = nx.single_source_shortest_path_length(G, s)
        d_true = lengths.get(t, -1)
        assert d == d_true
        horizon = d_true if d_true >= 0 else max(lengths.values())
        for v in range(g.n):
            if v in lengths and lengths[v] <= horizon:
                assert dist[v] == lengths[v]
                npaths = sum(1 for _ in nx.all_shortest_paths(G, s, v)) if v != s else 1
                assert sig[v] == npaths and ovf[v] == 0
            else:
                assert dist[v] == -1


def test_grid_sigma_closed_form():
    W, H = 9, 7
    g = I.grid_rewired(W, H, 0.0, 1)
    d, dist, sig, _ = O.Graph.of(g).sigma_bfs(0, W * H - 1)
    assert d == W + H - 2
    for v in range(W * H):
        x, y = v % W, v // W
        assert dist[v] == x + y and sig[v] == math.comb(x + y, x)


def test_tree_sigma_is_one():
    T = nx.random_labeled_tree(40, seed=2)
    g = nx_to_graph(T, directed=False)
    og = O.Graph.of(g)
    for s, t in [(0, 39), (5, 17), (12, 3)]:
        d, dist, sig, _ = og.sigma_bfs(s, t)
        assert d == nx.shortest_path_length(T, s, t)
        assert all(sig[v] == 1 for v in range(40) if dist[v] >= 0)


def _find_pair(n, seed, pred, limit=200000):
    for j in range(limit):
        s, t = O.pair(seed, j, n)
        if pred(s, t):
            return j, s, t
    raise AssertionError("no pair found")


def test_sigma_beyond_64_bits_is_exact():
    # 40x40 grid: corner to corner has C(78, 39) > 2^64 shortest paths
    W = 40
    g = I.grid_rewired(W, W, 0.0, 1)
    og = O.Graph.of(g)
    d, dist, sig, ovf = og.sigma_bfs(0, W * W - 1)
    assert sig[W * W - 1] == math.comb(78, 39) > 2**64 and ovf[W * W - 1] == 0
    # a sampled pair whose count exceeds 2^64 still yields a valid shortest path
    def big(s, t):
        dx, dy = abs(s % W - t % W), abs(s // W - t // W)
        return math.comb(dx + dy, dx) > 2**64
    j, s, t = _find_pair(W * W, 21, big)
    rc, s2, t2, dd, path = og.hyperedge(21, j)
    assert rc == O.OK and (s2, t2) == (s, t) and len(path) == dd - 1
    full = [s] + path + [t]
    for a, b in zip(full, full[1:]):
        assert abs(a % W - b % W) + abs(a // W - b // W) == 1


def test_sigma_beyond_128_bits_overflows():
    W = 70  # C(138, 69) > 2^128
    g = I.grid_rewired(W, W, 0.0, 1)
    og = O.Graph.of(g)
    d, dist, sig, ovf = og.sigma_bfs(0, W * W - 1)
    assert ovf[W * W - 1] == 1
    def huge(s, t):
        dx, dy = abs(s % W - t % W), abs(s // W - t // W)
        return math.comb(dx + dy, dx) >= 2**128
    j, s, t = _find_pair(W * W, 3, huge)
    assert og.hyperedge(3, j)[0] == O.EOVERFLOW
    def fits(s, t):
        dx, dy = abs(s % W - t % W), abs(s // W - t // W)
        return 2**100 < math.comb(dx + dy, dx) < 2**128
    j, s, t = _find_pair(W * W, 3, fits)
    assert og.hyperedge(3, j)[0] == O.OK


def test_star_complete_unreachable():
    star = O.Graph.of(nx_to_graph(nx.star_graph(7)))  # centre 0, leaves 1..7
    job = O.Job(star, 4, 4)
    job.sample(400)
    h = job.hypergraph()
    for j in range(400):
        mem = h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()
        leaves = h["s"][j] != 0 and h["t"][j] != 0
        assert mem == ([0] if leaves else [])
    # set betweenness of the centre is (n-2)/n: fraction of ordered pairs of leaves
    assert abs(np.mean(np.diff(h["hoff"])) - 6 / 8) < 0.07
    comp = O.Job(O.Graph.of(nx_to_graph(nx.complete_graph(6))), 4, 4)
    comp.sample(300)
    assert comp.hypergraph()["hoff"][-1] == 0
    dpath = O.Job(O.Graph.of(nx_to_graph(nx.path_graph(5, create_using=nx.DiGraph))), 4, 4)
    dpath.sample(300)
    hh = dpath.hypergraph()
    for j in range(300):
        s, t, d = hh["s"][j], hh["t"][j], hh["d"][j]
        assert d == (t - s if t > s else -1)
        assert (hh["hoff"][j + 1] - hh["hoff"][j]) == max(d - 1, 0)


@pytest.mark.parametrize("name,N", [("grid4x4", 120000), ("petersen", 60000), ("cycle8", 40000),
                                    ("ba20", 120000), ("digraph10", 60000)])
def test_path_frequencies_chi_square(name, N):
    graphs = {
        "grid4x4": I.grid_rewired(4, 4, 0.0, 1),
        "petersen": nx_to_graph(nx.petersen_graph()),
        "cycle8": nx_to_graph(nx.cycle_graph(8)),
        "ba20": I.ba(20, 2, 11),
        "digraph10": nx_to_graph(nx.gnp_random_graph(10, 0.3, seed=8, directed=True)),
    }
    g = graphs[name]
    G = graph_to_nx(g)
    n = g.n
    expect = {}
    for s in range(n):
        for t in range(n):
            if s == t:
                continue
            if not nx.has_path(G, s, t):
                expect[(s, t, ())] = 1.0 / (n * (n - 1))
                continue
            paths = list(nx.all_shortest_paths(G, s, t))
            for p in paths:
                expect[(s, t, tuple(p[1:-1]))] = 1.0 / (n * (n - 1) * len(paths))
    job = O.Job(O.Graph.of(g), 2024, 4)
    job.sample(N)
    h = job.hypergraph()
    obs = Counter()
    for j in range(N):
        obs[(int(h["s"][j]), int(h["t"][j]), tuple(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()))] += 1
    assert set(obs) <= set(expect)
    keys = sorted(expect)
    o = np.array([obs.get(k, 0) for k in keys], float)
    e = np.array([expect[k] * N for k in keys])
    assert abs(e.sum() - N) < 1e-6 * N
    assert stats.chisquare(o, e).pvalue > 1e-5


def exact_set_betweenness(G, n, S):
    """B(S) = 1/(n(n-1)) sum_{s != t} (shortest s-t paths with an interior node in S) / sigma_st."""
    S = set(S)
    tot = 0.0
    for s in range(n):
        for t in range(n):
            if s == t or not nx.has_path(G, s, t):
                continue
            paths = list(nx.all_shortest_paths(G, s, t))
            hit = sum(1 for p in paths if S & set(p[1:-1]))
            tot += hit / len(paths)
    return tot / (n * (n - 1))


def test_sample_estimate_within_hoeffding_of_exact_set_betweenness():
    g = I.ba(40, 2, 5)
    G = graph_to_nx(g)
    job = O.Job(O.Graph.of(g), 77, 4)
    m = 30000
    job.sample(m)
    h = job.hypergraph()
    members = [set(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()) for j in range(m)]
    deg = np.diff(g.off)
    for S in ([int(np.argmax(deg))], [0, 1, 2], [5, 17, 30, 39]):
        est = sum(1 for mm in members if mm & set(S)) / m
        exact = exact_set_betweenness(G, g.n, S)
        assert abs(est - exact) <= math.sqrt(math.log(2 / 1e-6) / (2 * m))


def test_work_tallies_match_networkx():
    g = I.ba(60, 3, 2)
    G = graph_to_nx(g)
    job = O.Job(O.Graph.of(g), 9, 4)
    job.sample(50)
    h = job.hypergraph()
    reached = arcs = 0
    deg = np.diff(g.off)
    for j in range(50):
        lengths = nx.single_source_shortest_path_length(G, int(h["s"][j]))
        d = int(h["d"][j])
        reached += sum(1 for v, l in lengths.items() if l < d)
        arcs += sum(int(deg[v]) for v, l in lengths.items() if l < d - 1)
    w = job.work()
    assert w[0] == reached and w[1] == arcs and w[3] == h["hoff"][-1]


def test_shards_by_sample_index_concatenate_to_the_whole():
    """Samples are functions of (seed, j): shards over disjoint index ranges, in order,
    give the same store as one job (the basis of sharded timing and of replicas)."""
    g = O.Graph.of(I.ba(300, 3, 2))
    whole = O.Job(g, 13, 4)
    whole.sample(500)
    ref = whole.hypergraph()
    parts = []
    for a, b in ((0, 170), (170, 171), (171, 500)):
        job = O.Job(g, 13, 4)
        job.sample_from(a, b - a)
        parts.append(job.hypergraph())
    assert np.concatenate([p["s"] for p in parts]).tolist() == ref["s"].tolist()
    assert np.concatenate([p["hmem"] for p in parts]).tolist() == ref["hmem"].tolist()
    lens = np.concatenate([np.diff(p["hoff"]) for p in parts])
    assert lens.tolist() == np.diff(ref["hoff"]).tolist()


def test_index_shards_in_worker_processes_equal_one_job():
    """Samples are functions of their index: ranges drawn in spawned worker processes and
    stored in index order give the single job's samples, and so its greedy and AMCERA."""
    from oracle import shards
    g = I.rmat(9, 8, seed=5)
    one = O.Job(O.Graph.of(g), 17, 12)
    one.sample(700)
    with shards.Pool(g, 2) as pool:
        merged = pool.job(17, 12, 700, chunk=128)
        picks = pool.hyperedges(17, [0, 5, 699])
    a, b = one.hypergraph(), merged.hypergraph()
    for key in ("hoff", "s", "t", "d"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["hmem"][: a["hoff"][-1]], b["hmem"][: b["hoff"][-1]])
    Sa, ca = one.greedy_cover(9)
    Sb, cb = merged.greedy_cover(9)
    assert Sa.tolist() == Sb.tolist() and ca == cb
    Ra, Wa, ba = one.mcera(9)
    Rb, Wb, bb = merged.mcera(9)
    assert np.array_equal(Ra, Rb) and Wa == Wb and ba == bb
    assert np.array_equal(one.rade_matrix()[0], merged.rade_matrix()[0])
    og = O.Graph.of(g)
    for j, r in picks.items():
        assert r == og.hyperedge(17, j)
