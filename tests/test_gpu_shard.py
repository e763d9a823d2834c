"""One sample split over shards on the GPU: the shard entry points and the driver.

Jobs with cen_job_set_ids(N, r) draw exactly the samples with ids r, r + N, ...
(their union is the single job's store); the shards' R and c sum to the single job's;
the top-k sums over a matrix equal cen_mcera's; and Algorithm 1 run over 2 or 3
shards in one process (the exchange is then a sum over the shards' device vectors)
equals cen_run and the oracle's run: set, coverage, sizes, rounds and log.  The
same driver over several processes is covered on CPU in test_shard_gloo.py.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")
from paper_2306_03651_gb300 import shard as SH  # noqa: E402


@pytest.mark.parametrize("N", [2, 3])
def test_shard_samples_rade_and_topk(N):
    g = I.rmat(12, 8, seed=3)
    gg = P.Graph.of(g)
    m, t, seed = 3001, 12, 7
    one = P.Job(gg, seed, t)
    one.sample(m)
    h1 = one.samples()
    Rnum1, Wnum1, b1 = one.mcera(9)
    R1, c1 = one.rade()
    Rsum = torch.zeros((t + 1, g.n), dtype=torch.int32, device="cuda")
    b = 0
    for r in range(N):
        job = P.Job(gg, seed, t)
        job.set_ids(N, r)
        cnt = SH.ids_below(m, N, r)
        job.sample(cnt // 2)
        job.sample(cnt - cnt // 2)
        h = job.samples()
        ids = np.arange(r, m, N)
        assert np.array_equal(h["s"], h1["s"][ids]) and np.array_equal(h["t"], h1["t"][ids])
        assert np.array_equal(h["d"], h1["d"][ids])
        for p, j in enumerate(ids):
            assert h["hmem"][h["hoff"][p]:h["hoff"][p + 1]].tolist() == \
                h1["hmem"][h1["hoff"][j]:h1["hoff"][j + 1]].tolist()
        buf = torch.empty((t + 1, g.n), dtype=torch.int32, device="cuda")
        b = max(b, job.shard_rade(buf))
        Rsum += buf
    assert np.array_equal(Rsum[:t].cpu().numpy(), R1) and np.array_equal(Rsum[t].cpu().numpy(), c1) and b == b1
    sums = one.shard_topk(Rsum, t + 1, 9)
    assert np.array_equal(sums[:t], Rnum1) and sums[t] == Wnum1
    with pytest.raises(P.CenError):
        one.set_ids(2, 0)  # the job already holds samples


@pytest.mark.parametrize("name,shards", [("ba2000", 2), ("rmat12", 3)])
def test_sharded_run_equals_one_job_and_the_oracle(name, shards):
    g = {"ba2000": I.ba(2000, 4, 1), "rmat12": I.rmat(12, 8, seed=3)}[name]
    gg = P.Graph.of(g)
    kw = dict(k=10, eps=0.05, delta=0.1, t=10, seed=1)
    one = P.run(gg, kw["k"], kw["eps"], kw["delta"], kw["t"], kw["seed"], m0=1000)
    sh = SH.run_sharded(gg, kw["k"], kw["eps"], kw["delta"], kw["t"], kw["seed"], m0=1000, shards=shards)
    ref = O.Graph.of(g).run(m0=1000, **kw)
    for r in (one, ref):
        assert sh["status"] == r["status"] == P.OK
        assert sh["S"].tolist() == r["S"].tolist() and sh["covered"] == r["covered"]
        assert sh["m_final"] == r["m_final"] and sh["rounds"] == r["rounds"]
        assert np.array_equal(sh["log"], r["log"])


def test_sharded_run_rmat18_equals_one_job():
    wl = I.rmat18_lcc()
    gg = P.Graph.of(wl.graph)
    one = P.run(gg, wl.k, 0.05, wl.delta, wl.t, wl.seed, m0=1000)
    sh = SH.run_sharded(gg, wl.k, 0.05, wl.delta, wl.t, wl.seed, m0=1000, shards=2)
    assert sh["status"] == one["status"] == P.OK
    assert sh["S"].tolist() == one["S"].tolist() and sh["covered"] == one["covered"]
    assert sh["m_final"] == one["m_final"] and np.array_equal(sh["log"], one["log"])
