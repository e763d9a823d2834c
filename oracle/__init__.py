"""CentRA oracle (ctypes binding) -- TEST INFRASTRUCTURE ONLY.

Plain single-threaded CPU CentRA (Algorithm 1 of Pellegrina, KDD'23, with the
set-betweenness sampler of Sec. 5) that the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, EOVERFLOW, ENOTCERTIFIED = 0, -1, -2, -4, -5
LOG_COLS = ("i", "m", "covered", "Rsum", "Wnum", "b", "C", "A", "w", "nu", "xi", "Rt", "R", "eta", "stop", "S_size")


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    u32, i32, i64, u64, dbl, vp = (ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_void_p)
    sig = {
        "orc_philox4x32_10": ([vp, vp, vp], None),
        "orc_uniform_below": ([u64, u64, u32, u64, u64, vp, vp], ctypes.c_int),
        "orc_pair": ([u64, u64, i32, vp, vp], None),
        "orc_sign_words": ([u64, u64, i32, vp], None),
        "orc_graph_new": ([i32, i64, vp, vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "orc_graph_free": ([vp], None),
        "orc_sigma_bfs": ([vp, i32, i32, vp, vp, vp, vp], i32),
        "orc_hyperedge": ([vp, u64, u64, vp, vp, vp, vp, vp], ctypes.c_int),
        "orc_job_new": ([vp, u64, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "orc_job_free": ([vp], None),
        "orc_job_sample": ([vp, u64], ctypes.c_int),
        "orc_job_sample_from": ([vp, u64, u64], ctypes.c_int),
        "orc_job_append": ([vp, u64, u64, vp, vp, vp, vp, vp], ctypes.c_int),
        "orc_job_m": ([vp], u64),
        "orc_job_members": ([vp], i64),
        "orc_job_copy": ([vp, vp, vp, vp, vp, vp], None),
        "orc_job_work": ([vp, vp], None),
        "orc_greedy_cover": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "orc_mcera": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "orc_rade_matrix": ([vp, vp, vp], ctypes.c_int),
        "orc_bounds": ([u64, u64, i64, i32, i64, i32, dbl, dbl, i32, vp], ctypes.c_int),
        "orc_run": ([vp, i32, dbl, dbl, i32, u64, u64, u64, vp, vp, vp, vp, vp, vp, i32], ctypes.c_int),
        "orc_run_ex": ([vp, i32, dbl, dbl, i32, u64, u64, u64, i32, dbl, i32, i32, i32, vp, vp, vp, vp, vp, vp,
                        i32], ctypes.c_int),
        "orc_job_new_space": ([vp, u64, i32, i32, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "orc_triangle_count": ([vp], i64),
        "orc_triangle_unrank": ([vp, i64, vp, vp, vp], ctypes.c_int),
        "orc_bounds_hedge": ([u64, u64, i32, i32, dbl, dbl, i32, vp], ctypes.c_int),
        "orc_schedule_guess": ([dbl, dbl, dbl, i32], dbl),
        "orc_schedule_next": ([i32, dbl, u64, u64, dbl, u64, dbl, dbl, i32], u64),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"{what}: oracle status {rc}")
        self.rc = rc


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform_below(seed: int, j: int, purpose: int, B: int):
    """Returns (value, rejected attempts) for B in [1, 2^128)."""
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    att = _load().orc_uniform_below(seed, j, purpose, B & (2**64 - 1), B >> 64, ctypes.byref(lo), ctypes.byref(hi))
    if att < 0:
        raise OracleError(att, "uniform_below")
    return (hi.value << 64) | lo.value, att


def pair(seed: int, j: int, n: int):
    s, t = ctypes.c_int32(), ctypes.c_int32()
    _load().orc_pair(seed, j, n, ctypes.byref(s), ctypes.byref(t))
    return s.value, t.value


def sign_words(seed: int, j: int, t: int) -> np.ndarray:
    out = np.zeros((t + 31) // 32, dtype=np.uint32)
    _load().orc_sign_words(seed, j, t, _p(out))
    return out


class Graph:
    def __init__(self, n, off, col, directed=False):
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.n = int(n)
        self.directed = bool(directed)
        h = ctypes.c_void_p()
        rc = _load().orc_graph_new(self.n, int(self.off[-1]), _p(self.off), _p(self.col), int(directed),
                                   ctypes.byref(h))
        if rc:
            raise OracleError(rc, "graph_new")
        self.h = h

    @classmethod
    def of(cls, g):
        return cls(g.n, g.off, g.col, g.directed)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_free(self.h)
            self.h = None

    def sigma_bfs(self, s: int, t: int):
        """Returns (d(s,t), dist[n], sigma[n] as Python ints, overflow flags[n])."""
        n = self.n
        dist = np.empty(n, np.int32)
        lo = np.empty(n, np.uint64)
        hi = np.empty(n, np.uint64)
        ovf = np.empty(n, np.uint8)
        d = _load().orc_sigma_bfs(self.h, s, t, _p(dist), _p(lo), _p(hi), _p(ovf))
        sig = [(int(h) << 64) | int(l) for l, h in zip(lo, hi)]
        return d, dist, sig, ovf

    def hyperedge(self, seed: int, j: int):
        """Returns (rc, s, t, d, path list)."""
        s, t, d, ln = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        path = np.empty(self.n, np.int32)
        rc = _load().orc_hyperedge(self.h, seed, j, ctypes.byref(s), ctypes.byref(t), ctypes.byref(d),
                                   ctypes.byref(ln), _p(path))
        return rc, s.value, t.value, d.value, path[: ln.value].tolist() if rc == 0 else []

    def triangle_count(self) -> int:
        return int(_load().orc_triangle_count(self.h))

    def triangle(self, r: int):
        u, v, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        rc = _load().orc_triangle_unrank(self.h, r, ctypes.byref(u), ctypes.byref(v), ctypes.byref(w))
        if rc:
            raise OracleError(rc, "triangle_unrank")
        return u.value, v.value, w.value

    def run(self, k, eps, delta, t, seed, m0=1000, m_cap=1 << 26, max_rounds=64, schedule=0, alpha=1.2, rule=0,
            space=0, kappa=0):
        """Algorithm 1.  schedule 0 doubling / 1 the paper's / 2 the paper's plus a predicted size;
        rule 0 CentRA / 1 HEDGE-P."""
        S = np.empty(k, np.int32)
        size, rounds = ctypes.c_int32(), ctypes.c_int32()
        cov, mf = ctypes.c_uint64(), ctypes.c_uint64()
        log = np.zeros((max_rounds, 16), np.float64)
        rc = _load().orc_run_ex(self.h, k, eps, delta, t, seed, m0, m_cap, schedule, alpha, rule, space, kappa, _p(S),
                                ctypes.byref(size), ctypes.byref(cov), ctypes.byref(mf), ctypes.byref(rounds),
                                _p(log), max_rounds)
        if rc not in (OK, ENOTCERTIFIED):
            raise OracleError(rc, "run")
        return dict(status=rc, S=S[: size.value].copy(), covered=cov.value, m_final=mf.value, rounds=rounds.value,
                    log=log[: rounds.value].copy())


SPACE_BETWEENNESS, SPACE_KPATH, SPACE_TRIANGLE = 0, 1, 2


class Job:
    def __init__(self, graph: Graph, seed: int, t: int, space: int = 0, kappa: int = 0):
        self.graph = graph
        self.seed = seed
        self.t = t
        h = ctypes.c_void_p()
        rc = _load().orc_job_new_space(graph.h, seed, t, space, kappa, ctypes.byref(h))
        if rc:
            raise OracleError(rc, "job_new")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_job_free(self.h)
            self.h = None

    @property
    def m(self) -> int:
        return int(_load().orc_job_m(self.h))

    def sample(self, m_new: int):
        rc = _load().orc_job_sample(self.h, m_new)
        if rc:
            raise OracleError(rc, "sample")

    def sample_from(self, j_first: int, count: int):
        """Append the samples with ids j_first .. j_first+count-1 (shards by sample index)."""
        rc = _load().orc_job_sample_from(self.h, j_first, count)
        if rc:
            raise OracleError(rc, "sample_from")

    def append(self, j_first: int, h: dict):
        """Store samples j_first.. that another job of the same graph and seed drew
        (dict(hoff, hmem, s, t, d), hoff starting at 0), e.g. in a worker process."""
        hoff = np.ascontiguousarray(h["hoff"], np.int64)
        count = len(hoff) - 1
        hmem = np.ascontiguousarray(h["hmem"], np.int32)
        arr = [np.ascontiguousarray(h[k][:count], np.int32) for k in ("s", "t", "d")]
        rc = _load().orc_job_append(self.h, j_first, count, _p(hoff), _p(hmem) if len(hmem) else None,
                                    *[_p(a) for a in arr])
        if rc:
            raise OracleError(rc, "append")

    def hypergraph(self):
        """Returns dict(hoff, hmem, s, t, d) as numpy arrays."""
        L = _load()
        m = self.m
        tot = int(L.orc_job_members(self.h))
        hoff = np.empty(m + 1, np.int64)
        hmem = np.empty(max(tot, 1), np.int32)
        s = np.empty(max(m, 1), np.int32)
        t = np.empty(max(m, 1), np.int32)
        d = np.empty(max(m, 1), np.int32)
        L.orc_job_copy(self.h, _p(hoff), _p(hmem), _p(s), _p(t), _p(d))
        return dict(hoff=hoff, hmem=hmem[:tot], s=s[:m], t=t[:m], d=d[:m])

    def work(self) -> np.ndarray:
        out = np.zeros(4, np.uint64)
        _load().orc_job_work(self.h, _p(out))
        return out

    def greedy_cover(self, k: int):
        S = np.empty(k, np.int32)
        size = ctypes.c_int32()
        cov = ctypes.c_uint64()
        rc = _load().orc_greedy_cover(self.h, k, _p(S), ctypes.byref(size), ctypes.byref(cov))
        if rc:
            raise OracleError(rc, "greedy_cover")
        return S[: size.value].copy(), cov.value

    def mcera(self, k: int):
        Rnum = np.empty(self.t, np.int64)
        W = ctypes.c_int64()
        b = ctypes.c_int32()
        rc = _load().orc_mcera(self.h, k, _p(Rnum), ctypes.byref(W), ctypes.byref(b))
        if rc:
            raise OracleError(rc, "mcera")
        return Rnum, W.value, b.value

    def rade_matrix(self):
        n, t = self.graph.n, self.t
        R = np.empty((n, t), np.int32)
        c = np.empty(n, np.int32)
        _load().orc_rade_matrix(self.h, _p(R), _p(c))
        return R, c


def bounds(covered, m, Rsum, t, Wnum, b, eps, delta, i):
    """Returns (stop, dict of C, A, w, nu, xi, Rt, R, eta)."""
    out = np.zeros(8, np.float64)
    stop = _load().orc_bounds(covered, m, Rsum, t, Wnum, b, eps, delta, i, _p(out))
    return bool(stop), dict(zip(("C", "A", "w", "nu", "xi", "Rt", "R", "eta"), out.tolist()))


def bounds_hedge(covered, m, n, k, eps, delta, i):
    """HEDGE-P: returns (stop, dict of C, L_U, nu_U, eta_U)."""
    out = np.zeros(4, np.float64)
    stop = _load().orc_bounds_hedge(covered, m, n, k, eps, delta, i, _p(out))
    return bool(stop), dict(zip(("C", "LU", "nuU", "etaU"), out.tolist()))


def schedule_guess(C, eps, delta, i) -> float:
    return float(_load().orc_schedule_guess(C, eps, delta, i))


def schedule_next(schedule, alpha, m0, m_prev, C_prev, eps, delta, i, m_pred=0) -> int:
    return int(_load().orc_schedule_next(schedule, alpha, m0, m_prev, C_prev, m_pred, eps, delta, i))
