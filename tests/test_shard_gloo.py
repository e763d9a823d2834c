"""One Algorithm-1 run with its sample split over shards: the driver's exchange logic
on CPU with two gloo ranks (world size 2, two shards per rank, so four shards).

Each shard is a host stand-in for a GPU job: it draws its samples by id with the
oracle (sample id = position * shards + index, as cen_job_set_ids maps them), and
computes gains, picks, covered counts, R and c and top-k sums by their plain
definitions.  The driver (paper_2306_03651_gb300/shard.py) sums gains and R matrices
over the shards and the ranks, takes the maximum b_H, and lets rank 0 decide the
stop.  The result must equal the single-process oracle's run bit for bit: the set,
its coverage, the sample sizes, the rounds and every column of the log, FP64
bounds included.  (The same driver runs on the GPU library in test_gpu_shard.py.)
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2306_03651_gb300 import shard as SH  # noqa: E402


class HostShard:
    """A shard whose samples are the oracle's, by id (test stand-in for a GPU job)."""

    def __init__(self, og, seed, t):
        self.og, self.seed, self.t, self.n = og, seed, t, og.n
        self.stride, self.offset = 1, 0
        self.H, self.sig = [], []

    def set_ids(self, stride, offset):
        assert not self.H
        self.stride, self.offset = stride, offset

    def sample(self, m_new):
        import oracle as O
        for p in range(len(self.H), len(self.H) + m_new):
            j = p * self.stride + self.offset
            rc, s, tt, d, path = self.og.hyperedge(self.seed, j)
            assert rc == O.OK
            self.H.append(list(path))
            w = O.sign_words(self.seed, j, self.t)
            self.sig.append([1 if (w[q >> 5] >> (q & 31)) & 1 else -1 for q in range(self.t)])

    def shard_greedy_begin(self):
        self.gain = np.zeros(self.n, np.int32)
        for h in self.H:
            for u in h:
                self.gain[u] += 1
        self.cov = np.zeros(len(self.H), bool)

    def shard_gains(self, buf):
        buf.copy_(torch.from_numpy(self.gain))

    def shard_pick(self, gains):
        g = gains.numpy()
        u = int(np.argmax(g))  # first maximum: the lowest id among the largest gains
        return (u, int(g[u])) if g[u] > 0 else (-1, 0)

    def shard_apply(self, u):
        newly = 0
        for s, h in enumerate(self.H):
            if not self.cov[s] and u in h:
                self.cov[s] = True
                newly += 1
                for x in h:
                    self.gain[x] -= 1
        return newly

    def shard_rade(self, buf):
        R = np.zeros((self.t + 1, self.n), np.int32)
        for h, sg in zip(self.H, self.sig):
            for u in h:
                R[: self.t, u] += sg
                R[self.t, u] += 1
        buf.copy_(torch.from_numpy(R))
        return max((len(h) for h in self.H), default=0)

    def shard_topk(self, vals, nrows, k):
        v = vals.numpy()
        return np.array([int(np.sort(r[r > 0])[::-1][:k].sum()) for r in v[:nrows]], np.int64)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


PARAMS = dict(k=4, eps=0.25, delta=0.1, t=6, seed=5, m0=200)


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2306_03651_gb300 import inputs as I
    og = O.Graph.of(I.ba(60, 2, 3))
    p = PARAMS
    r = SH.run_sharded(og, p["k"], p["eps"], p["delta"], p["t"], p["seed"], m0=p["m0"], m_cap=1 << 16, shards=2,
                       group=dist.group.WORLD, make_job=lambda g, seed, t: HostShard(og, seed, t),
                       device=torch.device("cpu"))
    out[rank] = (r["status"], r["S"].tolist(), r["covered"], r["m_final"], r["rounds"], r["log"].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_ids_below_deals_every_id_once():
    for m in (0, 1, 7, 8, 1000, 1001):
        for N in (1, 2, 3, 8):
            assert sum(SH.ids_below(m, N, r) for r in range(N)) == m
            assert all(SH.ids_below(m, N, r) == len(range(r, m, N)) for r in range(N))


def test_two_gloo_ranks_four_shards_equal_the_oracle_run():
    import oracle as O
    from paper_2306_03651_gb300 import inputs as I
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    p = PARAMS
    ref = O.Graph.of(I.ba(60, 2, 3)).run(k=p["k"], eps=p["eps"], delta=p["delta"], t=p["t"], seed=p["seed"],
                                         m0=p["m0"], m_cap=1 << 16)
    assert ref["status"] == O.OK and ref["rounds"] >= 2
    for rank in range(world):
        status, S, covered, m_final, rounds, log = out[rank]
        assert status == 0 and S == ref["S"].tolist() and covered == ref["covered"]
        assert m_final == ref["m_final"] and rounds == ref["rounds"]
        assert np.array_equal(np.array(log), ref["log"])  # FP64 bounds included, bit for bit
