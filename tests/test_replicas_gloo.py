"""Multi-process replica logic of bench.py on CPU (gloo, world size 2).

The path shards by independent replicas (samples are keyed by (seed, j)), so
N > 1 runs one replica per rank with a rank-specific seed and times the job by
the slowest rank.  Here two gloo ranks check the max-over-ranks reduction and
that their seeds give distinct, reproducible sample streams (CPU oracle)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_2306_03651_gb300 import inputs as I
    mx = bench.reduce_max(10.0 + rank, "cpu")
    g = O.Graph.of(I.ba(200, 3, 1))
    seed = bench.rank_seed(rank)
    pairs = [O.pair(seed, j, g.n) for j in range(64)]
    job = O.Job(g, seed, 4)
    job.sample(64)
    h = job.hypergraph()
    again = O.Job(g, seed, 4)
    again.sample(64)
    same = (again.hypergraph()["hmem"].tolist() == h["hmem"].tolist())
    gathered = [None] * world
    dist.all_gather_object(gathered, (seed, pairs))
    out[rank] = (mx, same, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        mx, same, gathered = out[rank]
        assert mx == 11.0 and same
        (s0, p0), (s1, p1) = gathered
        assert s0 != s1 and p0 != p1
