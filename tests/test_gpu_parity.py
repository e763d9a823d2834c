"""GPU parity: every step of the CUDA path against the CPU oracle, bit for bit.

Sampler (pairs, distances, path counts incl. the 128-bit range, backward
walk, hyper-edge store), incidence, greedyCover, sign words, AMCERA
numerators and Algorithm 1 end to end.  Small graphs span several waves and a
ragged last wave; the R-MAT scale-18 LCC workload is checked on sampled
outputs the oracle computes one by one, plus properties that hold at any size.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2306_03651_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ba2000_run.json")


def small_graphs():
    star = I.from_edges(9, [0] * 8, list(range(1, 9)), False)
    kn = 7
    e = np.array([(a, b) for a in range(kn) for b in range(a + 1, kn)], np.int32)
    comp = I.from_edges(kn, e[:, 0], e[:, 1], False)
    dpath = I.from_edges(6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], True)
    return {
        "ba2000": I.ba(2000, 4, 1),
        "ba300": I.ba(300, 3, 7),
        "rmat12_dir": I.rmat(12, 8, seed=3, directed=True, keep_lcc=False),
        "rmat12_lcc": I.rmat(12, 8, seed=3),
        "grid_rewired": I.grid_rewired(48, 48, 0.02, 5),
        "star": star,
        "complete": comp,
        "dpath": dpath,
    }


GRAPHS = small_graphs()


def oracle_samples(g, seed, m, t=10):
    og = O.Graph.of(g)
    job = O.Job(og, seed, t)
    job.sample(m)
    return og, job, job.hypergraph()


def assert_same_samples(a, b):
    for x in (a, b):  # the offsets end at the member total the job counted
        assert x["hoff"][-1] == len(x["hmem"])
    for key in ("hoff", "s", "t", "d"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["hmem"], b["hmem"])


@pytest.mark.parametrize("name", list(GRAPHS))
def test_sample_parity(name):
    g = GRAPHS[name]
    m = 2600 if g.n > 50 else 700
    _, _, ref = oracle_samples(g, 11, m)
    job = P.Job(P.Graph.of(g), 11, 10)
    job.sample(m)
    assert_same_samples(job.samples(), ref)


@pytest.mark.parametrize("name", ["ba300", "rmat12_dir", "grid_rewired", "dpath"])
def test_sample_parity_bit_parallel_only(name):
    """The bit-parallel sampler alone (the bidirectional one's fallback) matches too."""
    g = GRAPHS[name]
    m = 2600 if g.n > 50 else 700
    _, _, ref = oracle_samples(g, 11, m)
    job = P.Job(P.Graph.of(g), 11, 10)
    job.set_param(P.PARAM_SAMPLER, P.SAMPLER_WAVES)
    job.sample(m)
    assert_same_samples(job.samples(), ref)
    assert job.sampler_info()["slots"] == 0


@pytest.mark.parametrize("name", ["ba2000", "rmat12_dir", "grid_rewired"])
def test_bidirectional_search_deferral(name):
    """Balls larger than a 16-node queue go whole to the bit-parallel sampler; the store
    (members in the arena and in place) is still the oracle's."""
    g = GRAPHS[name]
    _, _, ref = oracle_samples(g, 17, 1500)
    job = P.Job(P.Graph.of(g), 17, 10)
    job.set_param(P.PARAM_BIDIR_QUEUE, 16)
    job.sample(700)
    job.sample(800)
    assert_same_samples(job.samples(), ref)
    info = job.sampler_info()
    assert info["deferred_search"] > 0 and info["slots"] > 0


@pytest.mark.parametrize("table", [0, 1024])
@pytest.mark.parametrize("name", ["ba2000", "rmat12_dir", "grid_rewired", "rmat12_lcc"])
def test_bidirectional_node_table_and_direct_words(name, table):
    """Node state in the large table only (small table 0), or in a 1,024-entry small table
    that many searches outgrow, moving to the large table mid-search: the oracle's samples
    either way."""
    g = GRAPHS[name]
    _, _, ref = oracle_samples(g, 29, 2000)
    job = P.Job(P.Graph.of(g), 29, 10)
    job.set_param(P.PARAM_BIDIR_TABLE, table)
    job.sample(2000)
    assert_same_samples(job.samples(), ref)
    info = job.sampler_info()
    assert info["migrated"] == 0 if table == 0 else (name != "grid_rewired" or info["migrated"] > 0)


@pytest.mark.parametrize("warps", [0, 1])
@pytest.mark.parametrize("name", ["ba2000", "rmat12_dir", "grid_rewired", "rmat12_lcc"])
def test_bidirectional_warp_searches(name, warps):
    """Samples searched by single warps, and by a second launch of whole CTAs when a level, the
    node count or the depth is too large for a warp (1), or searched by whole CTAs only (0):
    the oracle's samples either way, over two calls."""
    g = GRAPHS[name]
    _, _, ref = oracle_samples(g, 31, 2600)
    job = P.Job(P.Graph.of(g), 31, 10)
    job.set_param(P.PARAM_BIDIR_WARPS, warps)
    job.sample(1300)
    job.sample(1300)
    assert_same_samples(job.samples(), ref)
    if warps == 0:
        assert job.sampler_info()["escalated"] == 0


@pytest.mark.parametrize("warps", [0, 1])
def test_bidirectional_level_cap_deferral(warps):
    """A 5000-cycle: pairs far apart need more than a warp search's 64 levels on one side
    (handed to the CTA) and more than a CTA search's level cap (255), and are searched by the
    bit-parallel sampler."""
    n = 5000
    g = I.from_edges(n, np.arange(n), (np.arange(n) + 1) % n, False)
    _, _, ref = oracle_samples(g, 2, 300)
    job = P.Job(P.Graph.of(g), 2, 10)
    job.set_param(P.PARAM_BIDIR_WARPS, warps)
    job.sample(300)
    assert_same_samples(job.samples(), ref)
    info = job.sampler_info()
    assert info["deferred_search"] > 0
    assert info["escalated"] >= info["deferred_search"] if warps else info["escalated"] == 0
    assert ref["d"].max() > 2 * 255


def test_workspace_reuse_across_jobs():
    """Jobs that take a finished job's cached workspace (stale state words under later
    epochs), interleaved with jobs of another shape, and jobs after the cache is
    released, all draw the oracle's samples."""
    refs = {name: oracle_samples(GRAPHS[name], 23, 1200)[2] for name in ("ba300", "rmat12_lcc")}
    graphs = {name: P.Graph.of(GRAPHS[name]) for name in refs}
    for round_ in range(3):
        for name in ("ba300", "rmat12_lcc", "ba300"):
            job = P.Job(graphs[name], 23, 10)
            job.sample(1200)
            assert_same_samples(job.samples(), refs[name])
            job.close()
        if round_ == 1:
            P.release_cached()


def test_sample_split_invariance():
    g = GRAPHS["ba300"]
    _, _, ref = oracle_samples(g, 5, 1000)
    for splits in ([1000], [1, 63, 936], [64, 64, 200, 672], [999, 1]):
        job = P.Job(P.Graph.of(g), 5, 10)
        for s in splits:
            job.sample(s)
        assert_same_samples(job.samples(), ref)


def test_long_paths_in_the_first_round_fill_the_arena_without_deferral():
    """Cycle of 1,001 nodes: paths of about 250 interior nodes, while a job's first round sizes
    the member arena for 8 per sample.  The arena is resized from the walks' own total and the
    samples run again on the bidirectional sampler; none is left to the fallback, and the
    samples are the oracle's, in this round and the next.  Both frontiers of a cycle always
    cost the same, so the searches stay under the level cap only if ties grow the shallower
    side."""
    n = 1001
    src = np.arange(n, dtype=np.int32)
    g = I.from_edges(n, src, (src + 1) % n, False)
    seed, m1, m2 = 9, 6000, 3000
    _, _, ref = oracle_samples(g, seed, m1 + m2)
    job = P.Job(P.Graph.of(g), seed, 10)
    job.sample(m1)
    info = job.sampler_info()
    assert info["deferred_search"] == 0, info  # balanced on ties
    assert info["deferred_walk"] == 0, info  # the arena was resized, not overflowed
    assert job.size()[1] > 8 * m1 + (1 << 20)  # more members than the first round's arena held
    job.sample(m2)
    assert job.sampler_info()["deferred_walk"] == 0
    assert_same_samples(job.samples(), ref)


def hub_layers(directed: bool):
    """Layers Z0 -> P -> M -> H -> Z2 and Z1 -> M: sources in Z0 or Z1 reach Z2 through one of
    8 hubs H whose rows (about 1,040 arcs: 40 from M, 1,000 from Z2) are far longer than 8 times
    the cone level of M they draw from (33 or more nodes), so the walk takes its step at a hub
    over those cone nodes.  Directed: the hubs' long rows are in-rows (arcs Z2 -> H), and a
    candidate's arc into the hub is found in its out-row."""
    rng = np.random.default_rng(11)
    nZ0, nZ1, nP, nM, nH, nZ2 = 600, 600, 40, 64, 8, 2000
    Z0 = np.arange(nZ0)
    Z1 = nZ0 + np.arange(nZ1)
    Pl = nZ0 + nZ1 + np.arange(nP)
    M = Pl[-1] + 1 + np.arange(nM)
    H = M[-1] + 1 + np.arange(nH)
    Z2 = H[-1] + 1 + np.arange(nZ2)
    src, dst = [], []

    def link(a, b, k):
        for x in a:
            for y in rng.choice(b, size=k, replace=False):
                src.append(x)
                dst.append(y)
    link(Z0, Pl, 3)
    link(Z1, M, 40)
    link(Pl, M, 40)
    link(M, H, 5)
    for z in Z2:  # hub -> z for 4 hubs, and (directed) z -> 4 hubs
        for h in rng.choice(H, size=4, replace=False):
            src.append(h)
            dst.append(z)
        if directed:
            for h in rng.choice(H, size=4, replace=False):
                src.append(z)
                dst.append(h)
    n = int(Z2[-1]) + 1
    return I.from_edges(n, np.array(src), np.array(dst), directed), int(Z1[-1]) + 1, int(Z2[0])


@pytest.mark.parametrize("directed", [False, True])
def test_walk_step_over_the_cone_nodes_at_a_hub(directed):
    """Walk steps at hubs whose rows are much longer than the cone level they draw from: the
    step looks up the cone nodes' arcs into the hub and picks by the running path count in
    ascending id order, the oracle's pick for every sample."""
    g, left_end, right_start = hub_layers(directed)
    seed, m = 17, 4000
    _, _, ref = oracle_samples(g, seed, m)
    through_hub = np.sum((ref["s"] < left_end) & (ref["t"] >= right_start) & (ref["d"] >= 3))
    assert through_hub > 300
    for warps in (0, 1):
        job = P.Job(P.Graph.of(g), seed, 10)
        job.set_param(P.PARAM_BIDIR_WARPS, warps)
        job.sample(m)
        assert_same_samples(job.samples(), ref)


def test_path_counts_beyond_64_bits():
    """60x60 grid: pairs with C(dx+dy, dx) >= 2^64 shortest paths take the 128-bit re-run."""
    W = 60
    g = I.grid_rewired(W, W, 0.0, 1)
    seed, m = 21, 400
    big = 0
    for j in range(m):
        s, t = O.pair(seed, j, W * W)
        dx, dy = abs(s % W - t % W), abs(s // W - t // W)
        big += math.comb(dx + dy, dx) >= 2**64
    assert big > 0
    _, _, ref = oracle_samples(g, seed, m)
    job = P.Job(P.Graph.of(g), seed, 10)
    job.sample(m)
    assert_same_samples(job.samples(), ref)
    assert job.sampler_info()["deferred_walk"] >= big  # their walks go to the 128-bit re-run


def test_path_counts_beyond_128_bits_overflow():
    W = 70
    g = I.grid_rewired(W, W, 0.0, 1)
    seed = 3
    jbad = None
    for j in range(20000):
        s, t = O.pair(seed, j, W * W)
        dx, dy = abs(s % W - t % W), abs(s // W - t // W)
        if math.comb(dx + dy, dx) >= 2**128:
            jbad = j
            break
    assert jbad is not None
    job = P.Job(P.Graph.of(g), seed, 4)
    if jbad > 0:
        job.sample(jbad)
    with pytest.raises(P.CenError) as ei:
        job.sample(1)
    assert ei.value.rc == P.EOVERFLOW
    assert job.m == jbad  # the job is unchanged by the failed call


def incidence_rows(h, n):
    rows = [[] for _ in range(n)]
    for j in range(len(h["hoff"]) - 1):
        for u in h["hmem"][h["hoff"][j]:h["hoff"][j + 1]]:
            rows[u].append(j)
    return rows


@pytest.fixture(params=["cluster", "cluster8", "grid"])
def greedy_form(request, monkeypatch):
    """greedyCover as one thread-block cluster (16 CTAs where the device allows it, the default
    for these sizes), with the diagnostic CEN_GREEDY_CLUSTER=8 as one 8-CTA cluster (the
    portable size), or with CEN_GREEDY_GRID=1 as the cooperative grid kernel that graphs over
    921,600 nodes use."""
    monkeypatch.delenv("CEN_GREEDY_GRID", raising=False)
    monkeypatch.delenv("CEN_GREEDY_CLUSTER", raising=False)
    if request.param == "grid":
        monkeypatch.setenv("CEN_GREEDY_GRID", "1")
    elif request.param == "cluster8":
        monkeypatch.setenv("CEN_GREEDY_CLUSTER", "8")
    return request.param


@pytest.mark.parametrize("name", ["ba2000", "rmat12_dir", "grid_rewired"])
def test_greedy_incidence_mcera_parity(name, greedy_form):
    g = GRAPHS[name]
    m, t = 3000, 40
    og, ojob, ref = oracle_samples(g, 9, m, t)
    job = P.Job(P.Graph.of(g), 9, t)
    job.sample(m)
    for k in (1, 5, 17, 60):
        S, cov = job.greedy_cover(k)
        S2, cov2 = ojob.greedy_cover(k)
        assert S.tolist() == S2.tolist() and cov == cov2
    noff, nsamp = job.incidence()
    rows = incidence_rows(ref, g.n)
    for u in range(g.n):
        assert sorted(nsamp[noff[u]:noff[u + 1]].tolist()) == rows[u]
    words = job.signs()
    for j in range(0, m, 7):
        assert np.array_equal(words[j], O.sign_words(9, j, t))
    for k in (1, 10, 100):
        Rn, Wn, b = job.mcera(k)
        Rn2, Wn2, b2 = ojob.mcera(k)
        assert np.array_equal(Rn, Rn2) and Wn == Wn2 and b == b2
    R, c = job.rade()
    R2, c2 = ojob.rade_matrix()
    assert np.array_equal(R, R2.T) and np.array_equal(c, c2)


def test_run_matches_oracle_golden_on_ba2000():
    with open(GOLDEN) as f:
        gold = json.load(f)
    w = I.ba_2000()
    r = P.run(P.Graph.of(w.graph), w.k, w.eps, w.delta, w.t, w.seed, m0=w.m0)
    assert r["status"] == gold["status"]
    assert r["S"].tolist() == gold["S"]
    assert r["covered"] == gold["covered"] and r["m_final"] == gold["m_final"] and r["rounds"] == gold["rounds"]
    log = [[float.fromhex(x) for x in row] for row in gold["log_hex"]]
    assert np.array_equal(r["log"], np.array(log))


def test_run_not_certified_on_complete_graph():
    g = GRAPHS["complete"]
    r = P.run(P.Graph.of(g), 2, 0.1, 0.1, 4, 1, m0=100, m_cap=1600)
    ro = O.Graph.of(g).run(2, 0.1, 0.1, 4, 1, m0=100, m_cap=1600)
    assert r["status"] == P.ENOTCERTIFIED == ro["status"]
    assert r["m_final"] == ro["m_final"] == 1600 and r["covered"] == 0


@pytest.mark.parametrize("name,k,eps,t", [("ba300", 5, 0.2, 10), ("rmat12_lcc", 10, 0.1, 25),
                                          ("grid_rewired", 4, 0.15, 8)])
def test_paper_schedule_run_matches_oracle(name, k, eps, t):
    """Sec. 4.2 schedule (growth by alpha plus the optimistic guess): the sample sizes,
    every bound of every round, the picks and the status equal the oracle's."""
    g = GRAPHS[name]
    r = P.run(P.Graph.of(g), k, eps, 0.1, t, 11, m0=1000, schedule=P.SCHEDULE_PAPER, alpha=1.2)
    ro = O.Graph.of(g).run(k, eps, 0.1, t, 11, m0=1000, schedule=1, alpha=1.2)
    assert r["status"] == ro["status"] == P.OK
    assert r["rounds"] == ro["rounds"] and r["m_final"] == ro["m_final"]
    assert r["S"].tolist() == ro["S"].tolist() and r["covered"] == ro["covered"]
    assert np.array_equal(r["log"], ro["log"])
    b = P.run_batch([dict(graph=P.Graph.of(g), k=k, eps=eps, delta=0.1, t=t, seed=11, m0=1000,
                          schedule=P.SCHEDULE_PAPER, alpha=1.2)], nworkers=1)[0]
    assert b["status"] == P.OK and np.array_equal(b["log"], ro["log"])


def test_fixed_m_bounds_over_t_match_oracle():
    """Fixed-m rounds over t (the shape of the t sweep): AMCERA numerators and every FP64
    bound equal the oracle's for t from 1 to 500, where sign words span 1 to 16 words."""
    g = GRAPHS["ba2000"]
    m, k = 2500, 50
    og = O.Graph.of(g)
    pg = P.Graph.of(g)
    for t in (1, 10, 50, 100, 250, 500):
        ojob = O.Job(og, 31 + t, t)
        ojob.sample(m)
        job = P.Job(pg, 31 + t, t)
        job.sample(m)
        S, cov = job.greedy_cover(k)
        S2, cov2 = ojob.greedy_cover(k)
        assert S.tolist() == S2.tolist() and cov == cov2
        Rn, Wn, b = job.mcera(k)
        Rn2, Wn2, b2 = ojob.mcera(k)
        assert np.array_equal(Rn, Rn2) and Wn == Wn2 and b == b2
        assert P.bounds(cov, m, int(Rn.sum()), t, Wn, b, 0.05, 0.05, 1) == \
            O.bounds(cov, m, int(Rn2.sum()), t, Wn2, b2, 0.05, 0.05, 1)
        job.close()


@pytest.mark.parametrize("name,k,eps,t,schedule,rule", [
    ("ba300", 5, 0.2, 10, 0, 1), ("ba300", 5, 0.2, 10, 1, 1), ("ba300", 5, 0.2, 10, 2, 0),
    ("ba300", 5, 0.2, 10, 2, 1), ("rmat12_lcc", 10, 0.1, 25, 2, 0), ("rmat12_lcc", 10, 0.1, 25, 2, 1),
    ("grid_rewired", 4, 0.15, 8, 2, 0)])
def test_schedules_and_hedge_p_rule_match_oracle(name, k, eps, t, schedule, rule):
    """HEDGE-P (union-bound SD, Sec. 6) and the predicting schedule: every round's
    sample size and bounds, the picks and the status equal the oracle's."""
    g = GRAPHS[name]
    r = P.run(P.Graph.of(g), k, eps, 0.1, t, 5, m0=1000, schedule=schedule, alpha=1.2, rule=rule)
    ro = O.Graph.of(g).run(k, eps, 0.1, t, 5, m0=1000, schedule=schedule, alpha=1.2, rule=rule)
    assert r["status"] == ro["status"] == P.OK
    assert r["S"].tolist() == ro["S"].tolist() and r["m_final"] == ro["m_final"]
    assert np.array_equal(r["log"], ro["log"])
    if schedule == 2 and rule == 1:
        b = P.run_batch([dict(graph=P.Graph.of(g), k=k, eps=eps, delta=0.1, t=t, seed=5, m0=1000,
                              schedule=schedule, alpha=1.2, rule=rule)], nworkers=1)[0]
        assert np.array_equal(b["log"], ro["log"])


def test_run_rejects_bad_options():
    gg = P.Graph.of(GRAPHS["ba300"])
    for kw in (dict(schedule=P.SCHEDULE_PAPER, alpha=1.0), dict(schedule=3), dict(rule=2),
               dict(schedule=P.SCHEDULE_EXTRAPOLATE, alpha=0.5)):
        with pytest.raises(P.CenError) as ei:
            P.run(gg, 3, 0.1, 0.1, 4, 1, **kw)
        assert ei.value.rc == P.EINVAL


def test_run_argument_checks():
    gg = P.Graph.of(GRAPHS["ba300"])
    for kw in (dict(k=0), dict(eps=0.0), dict(eps=0.7), dict(delta=1.0), dict(t=0)):
        args = dict(k=3, eps=0.1, delta=0.1, t=4, seed=1)
        args.update(kw)
        with pytest.raises(P.CenError) as ei:
            P.run(gg, **args)
        assert ei.value.rc == P.EINVAL


def test_graph_load_rejects_malformed_and_accepts_device_arrays():
    torch = pytest.importorskip("torch")
    g = GRAPHS["ba300"]
    bad = g.col.copy()
    r0, r1 = g.off[5], g.off[6]
    bad[r0], bad[r0 + 1] = bad[r0 + 1], bad[r0]  # unsorted row
    with pytest.raises(P.CenError) as ei:
        P.Graph(g.n, g.off, bad, False)
    assert ei.value.rc == P.EINVAL
    loop = g.col.copy()
    loop[r0] = 5  # self-loop in row 5 (row stays sorted only if 5 < next; validation must still fail)
    with pytest.raises(P.CenError):
        P.Graph(g.n, g.off, loop, False)
    dg = P.Graph(g.n, torch.from_numpy(g.off).cuda(), torch.from_numpy(g.col).cuda(), False)
    job = P.Job(dg, 3, 8)
    job.sample(300)
    _, _, ref = oracle_samples(g, 3, 300, 8)
    assert_same_samples(job.samples(), ref)


def _csr(n, rows):
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], np.int32)
    return off, col


@pytest.mark.parametrize("case", ["ok", "ok_empty_rows", "id_high", "id_negative", "repeat", "descending",
                                  "self_loop_inside", "self_loop_first", "off_not_rising", "off0", "off_end"])
def test_graph_load_validation_cases(case):
    """A canonical CSR (rows strictly ascending, ids in [0, n), no self-loop, offsets rising from 0
    to nnz) loads; each single violation is rejected with CEN_EINVAL, wherever it sits."""
    n = 9
    rows = [[1, 4, 7], [], [0, 5], [], [1, 2, 6, 8], [0], [], [3, 8], [2]]
    off, col = _csr(n, rows)
    if case == "ok_empty_rows":
        rows = [[], [], [5], [], [], [], [], [], []]
        off, col = _csr(n, rows)
    elif case == "id_high":
        col[4] = n
    elif case == "id_negative":
        col[0] = -1
    elif case == "repeat":
        rows[4] = [1, 2, 2, 8]
        off, col = _csr(n, rows)
    elif case == "descending":
        rows[0] = [1, 7, 4]
        off, col = _csr(n, rows)
    elif case == "self_loop_inside":
        rows[4] = [1, 2, 4, 8]  # sorted, holds its own node
        off, col = _csr(n, rows)
    elif case == "self_loop_first":
        rows[2] = [2, 5]
        off, col = _csr(n, rows)
    elif case == "off_not_rising":
        off[2] = off[3] + 1  # row 2 ends before it starts
    elif case == "off0":
        off[0] = 1
    elif case == "off_end":
        off[-1] = off[-2] - 1  # the last row ends before it starts (nnz is taken from off[n])
    if case.startswith("ok"):
        gg = P.Graph(n, off, col, True)
        assert gg.nnz == len(col)
        roff, rcol = gg.csr()  # the graph as loaded
        assert np.array_equal(roff, off) and np.array_equal(rcol, col)
        return
    with pytest.raises(P.CenError) as ei:
        P.Graph(n, off, col, True)
    assert ei.value.rc == P.EINVAL


def test_stats_and_timing():
    g = GRAPHS["ba2000"]
    job = P.Job(P.Graph.of(g), 1, 10)
    job.set_timing(True)
    job.sample(2048)
    job.greedy_cover(10)
    job.mcera(10)
    st = job.stats()
    assert st["bidir"]["launches"] >= 1 and st["bidir"]["units"] > 0
    assert st["bidir"]["ms"] > 0 and st["bidir"]["timed"] == st["bidir"]["launches"]
    assert st["greedy"]["launches"] >= 1 and st["select"]["launches"] >= 1
    job.reset_stats()
    assert job.stats()["bidir"]["launches"] == 0
    waves = P.Job(P.Graph.of(g), 1, 10)
    waves.set_param(P.PARAM_SAMPLER, P.SAMPLER_WAVES)
    waves.set_timing(True)
    waves.sample(2048)
    st = waves.stats()
    assert st["pairs"]["launches"] >= 1 and st["walk"]["launches"] >= 1 and st["bidir"]["launches"] == 0
    assert st["expand_pull"]["launches"] + st["expand_push"]["launches"] >= 1
    assert st["walk"]["ms"] > 0 and st["walk"]["timed"] == st["walk"]["launches"]


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def rmat18():
    return I.rmat18_lcc()


def test_rmat18_sampled_parity_and_properties(rmat18):
    """R-MAT scale 18 LCC at the benchmark's wave size: sampled hyper-edges vs the
    oracle one by one; every hyper-edge is a shortest path's interior."""
    g = rmat18.graph
    m = 4096
    job = P.Job(P.Graph.of(g), rmat18.seed, rmat18.t)
    job.sample(m)
    h = job.samples()
    og = O.Graph.of(g)
    rng = np.random.default_rng(0)
    picks = sorted(set(rng.choice(m, 40, replace=False).tolist()) | {0, 2047, 2048, m - 1})
    for j in picks:
        rc, s, t, d, path = og.hyperedge(rmat18.seed, j)
        assert rc == O.OK
        assert (h["s"][j], h["t"][j], h["d"][j]) == (s, t, d)
        assert h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist() == path
    # properties at any size: connected graph, lengths d - 1, consecutive nodes adjacent
    assert np.all(h["d"] >= 1)
    assert np.array_equal(np.diff(h["hoff"]), np.maximum(h["d"] - 1, 0))
    def has_arc(a, b):
        row = g.col[g.off[a]:g.off[a + 1]]
        i = int(np.searchsorted(row, b))
        return i < len(row) and row[i] == b
    for j in range(0, m, 37):
        full = [h["s"][j]] + h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist() + [h["t"][j]]
        assert len(set(full)) == len(full)
        for a, b in zip(full, full[1:]):
            assert has_arc(a, b)
    # greedy at full size: picks and coverage consistent with the hyper-edges
    S, cov = job.greedy_cover(rmat18.k)
    mem = [set(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()) for j in range(m)]
    Sset = set(S.tolist())
    assert cov == sum(1 for x in mem if x & Sset)
    chosen, covered = [], np.zeros(m, bool)
    for u in S.tolist():
        gains = np.zeros(g.n, np.int64)
        for j in np.flatnonzero(~covered):
            for x in mem[j]:
                gains[x] += 1
        assert gains[u] == gains.max() and u == int(np.argmax(gains))
        for j in np.flatnonzero(~covered):
            if u in mem[j]:
                covered[j] = True
        chosen.append(u)
        if len(chosen) >= 5:
            break


@pytest.mark.parametrize("name", ["ba2000", "rmat12_lcc", "rmat12_dir"])
def test_cover_and_mcera_equals_the_two_calls(name):
    """greedyCover and the AMCERA side by side on two streams give what the two calls give, on a
    job whose sample grows between rounds (the incidence is rebuilt each time)."""
    g = GRAPHS[name]
    gg = P.Graph.of(g)
    a, b = P.Job(gg, 41, 12), P.Job(gg, 41, 12)
    for m in (900, 1700):
        a.sample(m)
        b.sample(m)
        for k in (1, 7, 25):
            S, cov, Rnum, Wnum, bh = a.cover_and_mcera(k)
            S2, cov2 = b.greedy_cover(k)
            Rnum2, Wnum2, bh2 = b.mcera(k)
            assert np.array_equal(S, S2) and cov == cov2
            assert np.array_equal(Rnum, Rnum2) and Wnum == Wnum2 and bh == bh2
