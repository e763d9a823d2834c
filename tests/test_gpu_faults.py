"""Failure handling, injected on the host: a device allocation that fails at
every possible point of graph upload, job creation, sampling (with concurrent
wave pipelines), greedy cover and AMCERA returns CEN_ENOMEM, leaves the job
unchanged and freeable, and the library keeps working afterwards."""
import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2306_03651_gb300")


def attempt(g):
    gg = P.Graph.of(g)
    job = P.Job(gg, 5, 12)
    job.tune(wave_words=2, wave_streams=3)
    job.sample(400)
    m_ok = job.m
    try:
        job.sample(900)
    except P.CenError as e:
        assert e.rc == P.ENOMEM and job.m == m_ok
        raise
    job.greedy_cover(6)
    job.mcera(6)
    return job


def test_injected_allocation_failures():
    g = I.ba(1500, 3, 4)
    failures = 0
    try:
        for n in range(1, 200):
            P.cen_debug_fail_alloc(n)
            try:
                attempt(g)
                break  # fewer than n allocations: nothing failed
            except P.CenError as e:
                assert e.rc == P.ENOMEM and "injected" in P.last_error()
                failures += 1
    finally:
        P.cen_debug_fail_alloc(0)
    assert failures >= 10
    job = attempt(g)  # disarmed: everything works and matches the oracle
    o = O.Job(O.Graph.of(g), 5, 12)
    o.sample(1300)
    h, oh = job.samples(), o.hypergraph()
    for key in ("hoff", "hmem", "s", "t", "d"):
        assert np.array_equal(h[key], oh[key])
