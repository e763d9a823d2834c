"""Algorithm 1 with one sample split over several shards (one per GPU).

Samples, their signs and their hyper-edges are functions of (seed, sample id)
(Sec. 5 sampleHEs, Alg. 1 sampleRadeVars), so round i's ids 0 .. m_i - 1 are
dealt to N shards by id modulo N (`cen_job_set_ids(N, r)`) and every shard
draws its own.  What a round needs from the whole sample adds up over the
shards: greedyCover's gains (Sec. 3.1) and the AMCERA's R_q^u and c_u
(Sec. 4.1) are sums over samples.  So per round:

* each shard appends its new samples (no exchange);
* greedyCover, one pick at a time: the shards' gain vectors are summed, the
  pick is the largest summed gain with the lowest id (the single-GPU rule),
  and every shard applies it to its own samples;
* the shards' R [t+1][n] matrices are summed, and the top-k sums of the rows
  of the sum give every Rnum and Wnum; b_H is the maximum over shards;
* the FP64 bounds and the stopping test of Alg. 1 (Thm. 4.4) run on the host
  of every process from the same integers; rank 0's decision is broadcast.

The result equals a single job's (`cen_run` with the doubling schedule and
CentRA's rule): same set, coverage, sample sizes and log.  A process may hold
several shards (its exchange is then a sum over them) and processes exchange
through a torch.distributed group (NCCL for CUDA tensors, or gloo).  The
shards themselves come from `make_job` (default: a library job on the current
CUDA device); the vector sums are the only work outside the library.
"""
from __future__ import annotations

import numpy as np

from . import cen as P


def ids_below(m: int, shards: int, index: int) -> int:
    """How many of the sample ids 0 .. m-1 are index modulo shards."""
    return max(0, (m - index + shards - 1) // shards)


def run_sharded(graph, k: int, eps: float, delta: float, t: int, seed: int, m0: int = 1000,
                m_cap: int = 1 << 30, shards: int = 1, group=None, make_job=None, device=None,
                max_rounds: int = 64) -> dict:
    """Algorithm 1 over `shards` shards in this process times the processes of `group`.

    Returns dict(status, S, covered, m_final, rounds, log) like ``cen.run`` (doubling
    schedule from m0, CentRA's stopping rule); every process gets the same result."""
    import torch

    a = 1.0 - np.exp(-1.0)
    if not (k >= 1 and t >= 1 and 0.0 < eps < a and 0.0 < delta < 1.0 and 1 <= m0 <= m_cap and shards >= 1):
        raise P.CenError(P.EINVAL, "run_sharded: need k >= 1, t >= 1, 0 < eps < 1-1/e, 0 < delta < 1, "
                                   "1 <= m0 <= m_cap, shards >= 1")
    dist = None
    world, rank = 1, 0
    if group is not None:
        import torch.distributed as dist
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    N = world * shards
    if make_job is None:
        make_job = P.Job
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    jobs = []
    for s in range(shards):
        job = make_job(graph, seed, t)
        job.set_ids(N, rank * shards + s)
        jobs.append(job)
    n = graph.n

    def exchange_sum(bufs):
        """Sum of the local shards' tensors, then over the processes (in place in bufs[0])."""
        tot = bufs[0]
        for b in bufs[1:]:
            tot += b
        if dist is not None:
            dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
        return tot

    def exchange_max(x: int) -> int:
        if dist is None:
            return x
        v = torch.tensor([x], dtype=torch.int64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX, group=group)
        return int(v.item())

    gains = [torch.empty(n, dtype=torch.int32, device=device) for _ in jobs]
    R = [torch.empty((t + 1, n), dtype=torch.int32, device=device) for _ in jobs]
    log = np.zeros((max_rounds, len(P.LOG_COLS)), np.float64)
    m_prev, m_i, i = 0, min(m0, m_cap), 0
    S: list[int] = []
    covered = 0
    status = P.ENOTCERTIFIED
    while True:
        i += 1
        for s, job in enumerate(jobs):
            idx = rank * shards + s
            job.sample(ids_below(m_i, N, idx) - ids_below(m_prev, N, idx))
        # greedyCover over the summed gains, one pick at a time
        for job in jobs:
            job.shard_greedy_begin()
        S, covered = [], 0
        for _ in range(k):
            for job, buf in zip(jobs, gains):
                job.shard_gains(buf)
            u, g = jobs[0].shard_pick(exchange_sum(gains))
            if g == 0:
                break
            S.append(u)
            covered += g
            for job in jobs:
                job.shard_apply(u)
        # AMCERA over the summed R and c
        b = 0
        for job, buf in zip(jobs, R):
            b = max(b, job.shard_rade(buf))
        b = exchange_max(b)
        sums = jobs[0].shard_topk(exchange_sum(R), t + 1, k)
        Rsum, Wnum = int(sums[:t].sum()), int(sums[t])
        stop, bd = P.bounds(covered, m_i, Rsum, t, Wnum, b, eps, delta, i)
        if dist is not None:  # rank 0 decides (every rank computed the same)
            flag = torch.tensor([int(stop)], dtype=torch.int32, device=device)
            dist.broadcast(flag, src=0, group=group)
            stop = bool(flag.item())
        if i <= max_rounds:
            log[i - 1] = [i, m_i, covered, Rsum, Wnum, b, bd["C"], bd["A"], bd["w"], bd["nu"], bd["xi"], bd["Rt"],
                          bd["R"], bd["eta"], float(stop), len(S)]
        if stop:
            status = P.OK
            break
        if 2 * m_i > m_cap:  # the next size would exceed the cap
            break
        m_prev, m_i = m_i, 2 * m_i
    return dict(status=status, S=np.array(S, np.int32), covered=covered, m_final=m_i, rounds=i,
                log=log[: min(i, max_rounds)].copy())
