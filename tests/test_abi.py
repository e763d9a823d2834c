"""CPU checks of the boundary: libcen.so loads, exports every function that
include/cen.h declares, rejects bad arguments without touching a GPU, and its
host FP64 bounds (Thm. 4.4, Alg. 1 stopping test) equal the oracle's
bit for bit."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import paper_2306_03651_gb300 as P


def test_library_exports_every_header_function():
    names = P.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(P._lib, n)]
    assert missing == []


def test_version_and_error_text():
    assert P.cen_version() >= 100
    assert isinstance(P.last_error(), str)


def test_bounds_rejects_bad_arguments():
    out = np.zeros(8)
    stop = ctypes.c_int32()
    for args in [(0, 0, 0, 10, 0, 0, 0.1, 0.1, 1),   # m = 0
                 (0, 10, 0, 0, 0, 0, 0.1, 0.1, 1),   # t = 0
                 (0, 10, 0, 5, 0, 0, 0.1, 1.5, 1),   # delta >= 1
                 (0, 10, 0, 5, 0, 0, 0.1, 0.1, 0)]:  # i = 0
        assert P.cen_bounds(*args, out.ctypes.data, ctypes.byref(stop)) == P.EINVAL
    assert "cen_bounds" in P.last_error()


def test_bounds_match_oracle_bit_for_bit():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        m = int(rng.integers(1, 10**8))
        cov = int(rng.integers(0, m + 1))
        t = int(rng.integers(1, 200))
        Rsum = int(rng.integers(0, t * m // 10 + 1))
        Wnum = int(rng.integers(0, 50 * m))
        b = int(rng.integers(0, 60))
        eps = float(rng.uniform(1e-4, 0.6))
        delta = float(rng.uniform(1e-6, 0.99))
        i = int(rng.integers(1, 40))
        s1, b1 = P.bounds(cov, m, Rsum, t, Wnum, b, eps, delta, i)
        s2, b2 = O.bounds(cov, m, Rsum, t, Wnum, b, eps, delta, i)
        assert s1 == s2
        for k in b1:
            assert b1[k] == b2[k] or (math.isnan(b1[k]) and math.isnan(b2[k])), k


def test_hedge_bounds_match_oracle_bit_for_bit():
    rng = np.random.default_rng(4)
    for _ in range(2000):
        m = int(rng.integers(1, 10**9))
        cov = int(rng.integers(0, m + 1))
        n = int(rng.integers(2, 10**8))
        k = int(rng.integers(1, 500))
        eps = float(rng.uniform(1e-4, 0.6))
        delta = float(rng.uniform(1e-6, 0.99))
        i = int(rng.integers(1, 40))
        assert P.bounds_hedge(cov, m, n, k, eps, delta, i) == O.bounds_hedge(cov, m, n, k, eps, delta, i)
    out = np.zeros(4)
    stop = ctypes.c_int32()
    assert P.cen_bounds_hedge(10, 100, 1, 3, 0.1, 0.1, 1, out.ctypes.data, ctypes.byref(stop)) == P.EINVAL


def test_null_handles_rejected():
    S = np.zeros(4, np.int32)
    size, cov = ctypes.c_int32(), ctypes.c_uint64()
    assert P.cen_greedy_cover(None, 4, S.ctypes.data, ctypes.byref(size), ctypes.byref(cov)) == P.EINVAL
    assert P.cen_sample(None, 10) == P.EINVAL
    h = ctypes.c_void_p()
    assert P.cen_job_create(None, 1, 4, None, ctypes.byref(h)) == P.EINVAL
    off = np.array([0, 1], np.int64)
    col = np.array([0], np.int32)
    assert P.cen_graph_load(off.ctypes.data, col.ctypes.data, 1, 1, 0, 0, None, ctypes.byref(h)) == P.EINVAL


def test_new_entry_points_check_arguments_before_any_device_work():
    S = np.zeros(4, np.int32)
    R = np.zeros(4, np.int64)
    size, cov, W, b = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_int64(), ctypes.c_int32()
    assert P.cen_cover_and_mcera(None, 4, S.ctypes.data, ctypes.byref(size), ctypes.byref(cov), R.ctypes.data,
                                 ctypes.byref(W), ctypes.byref(b)) == P.EINVAL
    off = np.array([0, 1, 1], np.int64)
    col = np.array([1], np.int32)
    h = ctypes.c_void_p()
    # unknown flag; SYMMETRIZE on a directed graph; n < 2 -- all rejected on the host
    assert P.cen_graph_load_ex(off.ctypes.data, col.ctypes.data, 2, 1, 0, 0, 8, None, ctypes.byref(h)) == P.EINVAL
    assert P.cen_graph_load_ex(off.ctypes.data, col.ctypes.data, 2, 1, 1, 0, P.GRAPH_SYMMETRIZE, None,
                               ctypes.byref(h)) == P.EINVAL
    assert P.cen_graph_load_ex(off.ctypes.data, col.ctypes.data, 1, 1, 0, 0, P.GRAPH_CANONICALIZE, None,
                               ctypes.byref(h)) == P.EINVAL
    assert "SYMMETRIZE" in P.last_error() or "n >= 2" in P.last_error()
    assert P.cen_graph_copy(None, off.ctypes.data, col.ctypes.data) == P.EINVAL
    # an allocator needs both functions; restoring the default needs none
    assert P.cen_set_allocator(ctypes.cast(P._ALLOC_FN(lambda n, s, c: None), ctypes.c_void_p), None, None) == P.EINVAL
    assert P.cen_set_allocator(None, None, None) == P.OK


def test_shard_and_result_entry_points_check_arguments_before_any_device_work():
    out = np.zeros(4, np.int64)
    u, g, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    newly = ctypes.c_uint64()
    assert P.cen_job_set_ids(None, 2, 0) == P.EINVAL
    assert P.cen_shard_greedy_begin(None) == P.EINVAL
    assert P.cen_shard_gains(None, None) == P.EINVAL
    assert P.cen_shard_pick(None, None, ctypes.byref(u), ctypes.byref(g)) == P.EINVAL
    assert P.cen_shard_apply(None, 0, ctypes.byref(newly)) == P.EINVAL
    assert P.cen_shard_rade(None, None, ctypes.byref(b)) == P.EINVAL
    assert P.cen_shard_topk(None, None, 2, 3, out.ctypes.data) == P.EINVAL
    res = P.cen_job_result()
    assert P.cen_run_result(None, None, ctypes.byref(res)) == P.EINVAL
    spec = P.cen_job_spec()
    assert P.cen_run_result(ctypes.byref(spec), None, ctypes.byref(res)) == P.EINVAL  # no S buffer
    assert "null" in P.last_error()
