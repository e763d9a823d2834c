"""Pins of the oracle's greedyCover (Sec. 3.1) and AMCERA numerators (Sec. 4.1, Alg. 1).

greedyCover: the (1-1/e) guarantee against brute force over all k-subsets,
step-by-step agreement with a set-based brute force argmax, submodularity of
coverage, early stop at zero gain.  AMCERA: the per-vector sup against
brute-force enumeration of node subsets, the invariants of Lemma
4.2 (exact expectation over all 2^m sign vectors on tiny
samples), parity / range / aggregation invariants of R.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

A = 1 - math.exp(-1)


def small_job(n=14, d=2, seed=3, m=60, t=6, jseed=5):
    g = O.Graph.of(I.ba(n, d, seed))
    job = O.Job(g, jseed, t)
    job.sample(m)
    return g, job


def members(job):
    h = job.hypergraph()
    return [set(h["hmem"][h["hoff"][j]:h["hoff"][j + 1]].tolist()) for j in range(job.m)]


def coverage(mem, S):
    S = set(S)
    return sum(1 for h in mem if h & S)


@pytest.mark.parametrize("seed,k", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 3)])
def test_greedy_guarantee_vs_brute_force(seed, k):
    g, job = small_job(n=12, seed=seed, m=50, jseed=seed)
    mem = members(job)
    S, cov = job.greedy_cover(k)
    assert cov == coverage(mem, S)
    opt = max(coverage(mem, c) for c in itertools.combinations(range(12), k))
    assert cov >= (1 - 1 / math.e) * opt
    assert cov <= opt


@pytest.mark.parametrize("seed", range(6))
def test_greedy_steps_match_set_argmax(seed):
    g, job = small_job(n=20, seed=seed + 10, m=80, jseed=seed)
    mem = members(job)
    k = 6
    S, cov = job.greedy_cover(k)
    chosen = []
    for _ in range(k):
        base = coverage(mem, chosen)
        gains = [coverage(mem, chosen + [u]) - base for u in range(20)]
        best = max(gains)
        if best == 0:
            break
        chosen.append(gains.index(best))  # index() = lowest id among ties
    assert S.tolist() == chosen
    assert cov == coverage(mem, chosen)


def test_greedy_stops_at_zero_gain():
    # star: every non-empty hyper-edge is {centre}; one pick covers everything
    star = O.Graph.of(I.from_edges(6, [0] * 5, [1, 2, 3, 4, 5], False))
    job = O.Job(star, 1, 3)
    job.sample(200)
    S, cov = job.greedy_cover(5)
    assert S.tolist() == [0]
    assert cov == sum(1 for h in members(job) if h)


def test_coverage_is_monotone_submodular():
    g, job = small_job(n=16, m=70)
    mem = members(job)
    rng = np.random.default_rng(0)
    for _ in range(300):
        T = set(rng.choice(16, rng.integers(0, 8), replace=False).tolist())
        S = set(x for x in T if rng.random() < 0.5)
        u = int(rng.integers(0, 16))
        if u in T:
            continue
        dS = coverage(mem, S | {u}) - coverage(mem, S)
        dT = coverage(mem, T | {u}) - coverage(mem, T)
        assert dS >= dT >= 0
        # f_S = min(1, sum_{u in S} f_u) for each hyper-edge
        for h in mem[:10]:
            assert int(bool(h & S)) == min(1, sum(1 for x in S if x in h))


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_rnum_is_the_modular_sup_by_enumeration(k):
    g, job = small_job(n=10, m=40, t=5)
    R, c = job.rade_matrix()
    Rnum, Wnum, b = job.mcera(k)
    for q in range(5):
        best = 0
        for size in range(0, k + 1):
            for S in itertools.combinations(range(10), size):
                best = max(best, sum(int(R[u, q]) for u in S))
        assert Rnum[q] == best
    wbest = max(sum(int(c[u]) for u in S) for S in itertools.combinations(range(10), min(k, 10)))
    assert Wnum == wbest
    assert b == max(len(h) for h in members(job))


def test_rade_matrix_invariants():
    g, job = small_job(n=30, m=300, t=40)
    R, c = job.rade_matrix()
    mem = members(job)
    # c_u counts the samples holding u
    for u in range(30):
        assert c[u] == sum(1 for h in mem if u in h)
    # |R| <= c and R = c (mod 2): each of the c_u terms is +-1
    assert np.all(np.abs(R) <= c[:, None])
    assert np.all((R - c[:, None]) % 2 == 0)
    # aggregating per sample instead of per node gives the same column sums
    col = np.zeros(40, np.int64)
    for j, h in enumerate(mem):
        w = O.sign_words(5, j, 40)
        sgn = np.array([1 if (w[q >> 5] >> (q & 31)) & 1 else -1 for q in range(40)])
        col += sgn * len(h)
    assert np.array_equal(R.sum(axis=0), col)


def test_rnum_monotone_concave_in_k():
    g, job = small_job(n=40, m=400, t=8)
    prev, prev_inc = None, None
    r1 = job.mcera(1)[0]
    for k in range(1, 12):
        r = job.mcera(k)[0]
        assert np.all(r <= k * r1)
        if prev is not None:
            inc = r - prev
            assert np.all(inc >= 0)
            if prev_inc is not None:
                assert np.all(inc <= prev_inc)
            prev_inc = inc
        prev = r


def test_lemma_expectappxratio_exact_expectation():
    """ERA(F_k) <= E_sigma[AMCERA(F_k)] <= k ERA(F_1), expectations exact over all 2^m sign vectors.

    Computed independently of the oracle's sign generator (the lemma is a property
    of the definitions): it pins the reading that the AMCERA sup is over the
    additive objective of individual nodes."""
    mem = [{0, 1}, {1}, {2, 3}, {0}, {3}, {1, 2}, set(), {0, 3}, {2}]
    n, m, k = 4, len(mem), 2
    subsets_k = [S for size in range(k + 1) for S in itertools.combinations(range(n), size)]
    era_k = era_1 = amcera = 0.0
    for bits in range(1 << m):
        sig = [1 if (bits >> s) & 1 else -1 for s in range(m)]
        era_k += max(sum(sig[s] for s in range(m) if mem[s] & set(S)) for S in subsets_k) / m
        era_1 += max([0] + [sum(sig[s] for s in range(m) if u in mem[s]) for u in range(n)]) / m
        r = sorted((sum(sig[s] for s in range(m) if u in mem[s]) for u in range(n)), reverse=True)
        amcera += sum(x for x in r[:k] if x > 0) / m
    era_k, era_1, amcera = era_k / 2**m, era_1 / 2**m, amcera / 2**m
    assert era_k <= amcera + 1e-12
    assert amcera <= k * era_1 + 1e-12
    assert era_1 <= era_k + 1e-12


def test_mcera_t1_all_plus_reduces_to_max_coverage():
    """Footnote of Sec. 3.2: with t = 1 and sigma = all ones the MCERA is max coverage / m,
    while the AMCERA's additive sup is the sum of the k largest c_u (>= coverage)."""
    g, job = small_job(n=10, m=40)
    mem = members(job)
    k = 3
    c = [sum(1 for h in mem if u in h) for u in range(10)]
    mcera = max(coverage(mem, S) for S in itertools.combinations(range(10), k))
    _, Wnum, _ = job.mcera(k)
    assert Wnum == sum(sorted(c, reverse=True)[:k]) >= mcera
