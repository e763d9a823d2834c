"""GPU parity of the kappa-path and triangle hyper-edge spaces (Sec. 2) against the
oracle, sample by sample, and of Algorithm 1 run in those spaces."""
import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2306_03651_gb300")

GRAPHS = {
    "ba300": I.ba(300, 3, 7),
    "rmat12_lcc": I.rmat(12, 8, seed=3),
    "rmat12_dir": I.rmat(12, 8, seed=3, directed=True, keep_lcc=False),
    "grid_rewired": I.grid_rewired(48, 48, 0.02, 5),
}


def same(job, ojob):
    a, b = job.samples(), ojob.hypergraph()
    for key in ("hoff", "s", "t", "d", "hmem"):
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("kappa", [1, 4, 16])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_kpath_parity(name, kappa):
    g = GRAPHS[name]
    job = P.Job(P.Graph.of(g), 13, 8, space=P.SPACE_KPATH, kappa=kappa)
    ojob = O.Job(O.Graph.of(g), 13, 8, space=O.SPACE_KPATH, kappa=kappa)
    for m in (1, 700, 2300):
        job.sample(m)
        ojob.sample(m)
    same(job, ojob)
    Rn, Wn, b = job.mcera(10)
    Rn2, Wn2, b2 = ojob.mcera(10)
    assert np.array_equal(Rn, Rn2) and Wn == Wn2 and b == b2 <= kappa


def test_kpath_two_pass_when_the_walk_buffer_would_be_large():
    """300,000 walks of kappa = 1024 would stage 1.2 GB: the walks then run twice (lengths,
    then members in place).  A star keeps them short; the samples are still the oracle's."""
    n = 1001
    star = I.from_edges(n, [0] * (n - 1), list(range(1, n)), False)
    m = 300000
    job = P.Job(P.Graph.of(star), 7, 4, space=P.SPACE_KPATH, kappa=1024)
    job.sample(m)
    ojob = O.Job(O.Graph.of(star), 7, 4, space=O.SPACE_KPATH, kappa=1024)
    ojob.sample(m)
    same(job, ojob)


@pytest.mark.parametrize("name", ["ba300", "rmat12_lcc", "ba2000"])
def test_triangle_parity(name):
    g = GRAPHS[name] if name in GRAPHS else I.ba(2000, 4, 1)
    og = O.Graph.of(g)
    job = P.Job(P.Graph.of(g), 17, 8, space=P.SPACE_TRIANGLE)
    ojob = O.Job(og, 17, 8, space=O.SPACE_TRIANGLE)
    for m in (5, 3000):
        job.sample(m)
        ojob.sample(m)
    same(job, ojob)
    S, cov = job.greedy_cover(7)
    S2, cov2 = ojob.greedy_cover(7)
    assert S.tolist() == S2.tolist() and cov == cov2


@pytest.mark.parametrize("space,kappa", [(1, 5), (2, 0)])
def test_run_in_other_spaces_matches_oracle(space, kappa):
    g = GRAPHS["rmat12_lcc"]
    r = P.run(P.Graph.of(g), 10, 0.1, 0.1, 16, 21, m0=1000, schedule=P.SCHEDULE_EXTRAPOLATE, space=space, kappa=kappa)
    ro = O.Graph.of(g).run(10, 0.1, 0.1, 16, 21, m0=1000, schedule=2, space=space, kappa=kappa)
    assert r["status"] == ro["status"] == P.OK
    assert r["S"].tolist() == ro["S"].tolist() and np.array_equal(r["log"], ro["log"])


def test_spaces_reject_bad_arguments():
    gg = P.Graph.of(GRAPHS["ba300"])
    for kw in (dict(space=3), dict(space=P.SPACE_KPATH, kappa=0), dict(space=P.SPACE_KPATH, kappa=1025)):
        with pytest.raises(P.CenError) as ei:
            P.Job(gg, 1, 4, **kw)
        assert ei.value.rc == P.EINVAL
    with pytest.raises(P.CenError):
        P.Job(P.Graph.of(GRAPHS["rmat12_dir"]), 1, 4, space=P.SPACE_TRIANGLE)
    tree = I.from_edges(5, [0, 0, 1, 1], [1, 2, 3, 4], False)
    for g in (tree, GRAPHS["grid_rewired"]):  # no triangle: both sides reject the space
        assert O.Graph.of(g).triangle_count() == 0
        with pytest.raises(P.CenError):
            P.Job(P.Graph.of(g), 1, 4, space=P.SPACE_TRIANGLE)
