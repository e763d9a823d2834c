"""Pins of the oracle's other hyper-edge spaces (Sec. 2: kappa-path and triangle
centralities, on which CentRA works unchanged, Sec. 4.2 remark).

kappa-path: the exact law of (s, l, walk) by enumerating every walk of the process on
tiny graphs, against sampled frequencies (chi-square), plus the walk invariants.
Triangle: the count against networkx, the unranking as a bijection onto the
lexicographically ordered triangles, and uniformity (chi-square).
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2306_03651_gb300 import inputs as I

nx = pytest.importorskip("networkx")


def nx_graph(g):
    G = nx.DiGraph() if g.directed else nx.Graph()
    G.add_nodes_from(range(g.n))
    for v in range(g.n):
        for w in g.col[g.off[v]:g.off[v + 1]]:
            G.add_edge(v, int(w))
    return G


def kpath_law(g, kappa):
    """P(s, l, walk) of the kappa-path process, by enumeration."""
    law = {}
    nbrs = {v: [int(w) for w in g.col[g.off[v]:g.off[v + 1]]] for v in range(g.n)}

    def rec(s, l, walk, p):
        cur = walk[-1] if walk else s
        if len(walk) == l:
            law[(s, l, tuple(walk))] = law.get((s, l, tuple(walk)), 0) + p
            return
        free = [w for w in nbrs[cur] if w != s and w not in walk]
        if not free:
            law[(s, l, tuple(walk))] = law.get((s, l, tuple(walk)), 0) + p
            return
        for w in free:
            rec(s, l, walk + [w], p / len(free))

    for s in range(g.n):
        for l in range(1, kappa + 1):
            rec(s, l, [], 1.0 / (g.n * kappa))
    return law


@pytest.mark.parametrize("name,kappa,N", [("petersen", 3, 60000), ("digraph", 2, 40000), ("ba12", 4, 80000)])
def test_kpath_walk_law_chi_square(name, kappa, N):
    graphs = {
        "petersen": I.from_edges(*_edges(nx.petersen_graph()), False),
        "digraph": I.from_edges(*_edges(nx.gnp_random_graph(7, 0.35, seed=3, directed=True)), True),
        "ba12": I.ba(12, 2, 4),
    }
    g = graphs[name]
    law = kpath_law(g, kappa)
    assert abs(sum(law.values()) - 1) < 1e-12
    job = O.Job(O.Graph.of(g), 31, 4, space=O.SPACE_KPATH, kappa=kappa)
    job.sample(N)
    h = job.hypergraph()
    obs = Counter()
    for j in range(N):
        obs[(int(h["s"][j]), int(h["t"][j]), tuple(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()))] += 1
    assert set(obs) <= set(law)
    keys = sorted(law)
    o = np.array([obs.get(k, 0) for k in keys], float)
    e = np.array([law[k] * N for k in keys])
    assert stats.chisquare(o, e).pvalue > 1e-5


def _edges(G):
    G = nx.convert_node_labels_to_integers(G)
    e = np.array(list(G.edges()), dtype=np.int32)
    return G.number_of_nodes(), e[:, 0], e[:, 1]


def test_kpath_walk_invariants():
    g = I.rmat(9, 6, seed=2)
    kappa = 6
    job = O.Job(O.Graph.of(g), 5, 4, space=O.SPACE_KPATH, kappa=kappa)
    job.sample(3000)
    h = job.hypergraph()
    adj = [set(g.col[g.off[v]:g.off[v + 1]].tolist()) for v in range(g.n)]
    for j in range(3000):
        s, l, steps = int(h["s"][j]), int(h["t"][j]), int(h["d"][j])
        walk = h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()
        assert 1 <= l <= kappa and steps == len(walk) <= l
        assert s not in walk and len(set(walk)) == len(walk)
        full = [s] + walk
        assert all(b in adj[a] for a, b in zip(full, full[1:]))
        if steps < l:  # stopped early: every neighbour of the last node is on the walk
            assert adj[full[-1]] <= set(full)


def test_triangles_count_and_unranking_is_the_sorted_list():
    for g in (I.ba(40, 3, 1), I.rmat(8, 8, seed=4), I.grid_rewired(6, 6, 0.3, 2)):
        G = nx_graph(g)
        tris = sorted(tuple(sorted(c)) for c in nx.enumerate_all_cliques(G) if len(c) == 3)
        og = O.Graph.of(g)
        assert og.triangle_count() == len(tris) == sum(nx.triangles(G).values()) // 3
        assert [og.triangle(r) for r in range(len(tris))] == tris


def test_triangle_sampling_is_uniform_and_ordered():
    g = I.ba(30, 3, 7)
    og = O.Graph.of(g)
    T = og.triangle_count()
    N = 40 * T
    job = O.Job(og, 9, 4, space=O.SPACE_TRIANGLE)
    job.sample(N)
    h = job.hypergraph()
    assert np.array_equal(np.diff(h["hoff"]), np.full(N, 3))
    mem = h["hmem"].reshape(-1, 3)
    assert (mem[:, 0] < mem[:, 1]).all() and (mem[:, 1] < mem[:, 2]).all()
    assert np.array_equal(mem, np.stack([h["s"], h["t"], h["d"]], 1))
    cnt = Counter(map(tuple, mem.tolist()))
    assert len(cnt) == T
    assert stats.chisquare(np.array([cnt[og.triangle(r)] for r in range(T)], float)).pvalue > 1e-5


def test_spaces_reject_bad_arguments():
    g = O.Graph.of(I.ba(30, 2, 1))
    for kw in (dict(space=3), dict(space=O.SPACE_KPATH, kappa=0)):
        with pytest.raises(O.OracleError):
            O.Job(g, 1, 4, **kw)
    tree = O.Graph.of(I.from_edges(5, [0, 0, 1, 1], [1, 2, 3, 4], False))
    with pytest.raises(O.OracleError):
        O.Job(tree, 1, 4, space=O.SPACE_TRIANGLE)  # no triangle to draw
    dg = O.Graph.of(I.from_edges(3, [0, 1, 2], [1, 2, 0], True))
    with pytest.raises(O.OracleError):
        O.Job(dg, 1, 4, space=O.SPACE_TRIANGLE)  # undirected graphs only


@pytest.mark.parametrize("space,kappa", [(O.SPACE_KPATH, 4), (O.SPACE_TRIANGLE, 0)])
def test_run_certifies_in_other_spaces(space, kappa):
    """Algorithm 1 is oblivious to sampleHEs: the loop certifies; the certified set reaches
    (1 - 1/e - eps) of the exact optimum of the space's coverage on a tiny graph."""
    g = I.ba(12, 3, 5)
    og = O.Graph.of(g)
    k, eps = 2, 0.3
    r = og.run(k=k, eps=eps, delta=0.1, t=10, seed=4, m0=1000, space=space, kappa=kappa)
    assert r["status"] == O.OK
    if space == O.SPACE_TRIANGLE:
        tris = [og.triangle(q) for q in range(og.triangle_count())]
        cov = lambda S: sum(1 for tr in tris if set(tr) & set(S)) / len(tris)
    else:
        law = kpath_law(g, kappa)
        cov = lambda S: sum(p for (s, l, walk), p in law.items() if set(walk) & set(S))
    opt = max(cov(S) for S in itertools.combinations(range(g.n), k))
    assert cov(r["S"]) >= (1 - 1 / math.e - eps) * opt
