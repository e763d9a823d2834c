"""ctypes binding of libcen.so (include/cen.h), the GB300 CentRA library.

Argument marshalling only: every step of the method runs in the CUDA library.
The raw C entry points are exported under their C names (``cen_sample`` ...);
``Graph``, ``Job``, ``run`` and ``bounds`` wrap them with numpy / torch
arguments.  Streams default to torch's current CUDA stream.

Importing this module loads ``libcen.so``, compiling it with nvcc first when
it is absent; if that fails the import raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcen.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cen.h")

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ENOTCERTIFIED = 0, -1, -2, -3, -4, -5
PARAM_WAVE_WORDS, PARAM_WAVE_STREAMS, PARAM_PUSH_RATIO, PARAM_LEVEL_BUDGET = 1, 2, 3, 4
PARAM_SAMPLER, PARAM_BIDIR_BUDGET, PARAM_BIDIR_QUEUE, PARAM_BIDIR_TABLE, PARAM_BIDIR_WARPS = 5, 6, 7, 8, 9
SAMPLER_BIDIR, SAMPLER_WAVES = 0, 1
SCHEDULE_DOUBLING, SCHEDULE_PAPER, SCHEDULE_EXTRAPOLATE = 0, 1, 2
RULE_CENTRA, RULE_HEDGE_P = 0, 1
SPACE_BETWEENNESS, SPACE_KPATH, SPACE_TRIANGLE = 0, 1, 2
GRAPH_CANONICALIZE, GRAPH_SYMMETRIZE = 1, 2
LOG_COLS = ("i", "m", "covered", "Rsum", "Wnum", "b", "C", "A", "w", "nu", "xi", "Rt", "R", "eta", "stop", "S_size")
NKCLASS = 24


class CenError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"{msg} (status {rc})")
        self.rc = rc


class cen_run_opts(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("rule", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("space", ctypes.c_int32), ("kappa", ctypes.c_int32)]


class cen_job_spec(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("k", ctypes.c_int32), ("t", ctypes.c_int32), ("eps", ctypes.c_double),
                ("delta", ctypes.c_double), ("seed", ctypes.c_uint64), ("m0", ctypes.c_uint64),
                ("m_cap", ctypes.c_uint64), ("opts", cen_run_opts)]


class cen_job_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("S_size", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("covered", ctypes.c_uint64), ("m_final", ctypes.c_uint64),
                ("S", ctypes.c_void_p), ("log", ctypes.c_void_p), ("start_s", ctypes.c_double),
                ("end_s", ctypes.c_double)]


class cen_kstat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("timed", ctypes.c_uint64), ("units", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        from . import _build
        try:
            _build.build()
        except Exception as e:  # no CUDA library means no product path
            raise ImportError(f"libcen.so is missing and could not be built: {e}") from e
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, u64, dbl, vp, ip = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_int)
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "cen_version": ([], ip),
        "cen_last_error": ([], ctypes.c_char_p),
        "cen_graph_load": ([vp, vp, i32, i64, ip, ip, vp, pvp], ip),
        "cen_graph_load_ex": ([vp, vp, i32, i64, ip, ip, ip, vp, pvp], ip),
        "cen_cover_and_mcera": ([vp, i32, vp, vp, vp, vp, vp, vp], ip),
        "cen_graph_copy": ([vp, vp, vp], ip),
        "cen_graph_free": ([vp], ip),
        "cen_graph_info": ([vp, vp, vp, vp], ip),
        "cen_job_create": ([vp, u64, i32, vp, pvp], ip),
        "cen_job_free": ([vp], ip),
        "cen_job_size": ([vp, vp, vp], ip),
        "cen_sample": ([vp, u64], ip),
        "cen_greedy_cover": ([vp, i32, vp, vp, vp], ip),
        "cen_mcera": ([vp, i32, vp, vp, vp], ip),
        "cen_bounds": ([u64, u64, i64, i32, i64, i32, dbl, dbl, i32, vp, vp], ip),
        "cen_run": ([vp, i32, dbl, dbl, i32, u64, u64, u64, vp, vp, vp, vp, vp, vp, vp, i32], ip),
        "cen_run_ex": ([vp, i32, dbl, dbl, i32, u64, u64, u64, vp, vp, vp, vp, vp, vp, vp, vp, i32], ip),
        "cen_bounds_hedge": ([u64, u64, i32, i32, dbl, dbl, i32, vp, vp], ip),
        "cen_job_copy_samples": ([vp, vp, vp, vp, vp, vp], ip),
        "cen_job_copy_incidence": ([vp, vp, vp], ip),
        "cen_job_copy_rade": ([vp, vp, vp], ip),
        "cen_job_copy_signs": ([vp, vp], ip),
        "cen_job_set_timing": ([vp, ip], ip),
        "cen_job_stats": ([vp, vp, vp], ip),
        "cen_job_sampler_info": ([vp, vp, vp, vp, vp, vp], ip),
        "cen_job_create_space": ([vp, u64, i32, i32, i32, vp, ctypes.POINTER(vp)], ip),
        "cen_release_cached": ([], ip),
        "cen_set_allocator": ([vp, vp, vp], ip),
        "cen_job_reset_stats": ([vp], ip),
        "cen_topk_positive_sum_noalloc": ([vp, i64, i32, i32, vp, vp], ip),
        "cen_run_batch": ([vp, i32, i32, vp], ip),
        "cen_run_result": ([vp, vp, vp], ip),
        "cen_job_set_param": ([vp, i32, dbl], ip),
        "cen_graph_set_param": ([vp, i32, dbl], ip),
        "cen_debug_fail_alloc": ([i64], ip),
        "cen_job_set_ids": ([vp, u64, u64], ip),
        "cen_shard_greedy_begin": ([vp], ip),
        "cen_shard_gains": ([vp, vp], ip),
        "cen_shard_pick": ([vp, vp, vp, vp], ip),
        "cen_shard_apply": ([vp, i32, vp], ip),
        "cen_shard_rade": ([vp, vp, vp], ip),
        "cen_shard_topk": ([vp, vp, i32, i32, vp], ip),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
        globals()[name] = f
    return lib


_lib = _load()


def header_functions() -> list[str]:
    """Names of the functions declared in include/cen.h."""
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cen_[a-z0-9_]+)\s*\(", src)))


def last_error() -> str:
    return (_lib.cen_last_error() or b"").decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise CenError(rc, f"{what}: {last_error()}")


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def current_stream():
    """torch's current CUDA stream handle (or None when torch/CUDA is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return None


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class Graph:
    """Device-resident canonical CSR graph (``cen_graph_load``)."""

    def __init__(self, n: int, off, col, directed: bool = False, stream=None, flags: int = 0):
        """flags: GRAPH_CANONICALIZE / GRAPH_SYMMETRIZE (``cen_graph_load_ex``); 0 takes a canonical CSR as is."""
        self.n = int(n)
        self.directed = bool(directed)
        self.stream = stream if stream is not None else current_stream()
        if _is_torch_cuda(off):
            on_dev, poff, pcol = 1, off.data_ptr(), col.data_ptr()
            nnz = int(col.numel())
            self._keep = (off, col)
        else:
            off = np.ascontiguousarray(off, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            on_dev, poff, pcol = 0, _p(off), _p(col)
            nnz = int(off[-1])
            self._keep = (off, col)
        h = ctypes.c_void_p()
        _check(_lib.cen_graph_load_ex(poff, pcol, self.n, nnz, int(directed), on_dev, int(flags), self.stream,
                                      ctypes.byref(h)), "cen_graph_load")
        self.h = h
        self._keep = None
        kept = ctypes.c_int64()
        _check(_lib.cen_graph_info(self.h, None, ctypes.byref(kept), None), "cen_graph_info")
        self.nnz = int(kept.value)

    def csr(self):
        """The device graph's CSR (off int64[n+1], col int32[nnz]) as host arrays (``cen_graph_copy``)."""
        off = np.zeros(self.n + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        _check(_lib.cen_graph_copy(self.h, _p(off), _p(col)), "cen_graph_copy")
        return off, col[:self.nnz]

    @classmethod
    def of(cls, g, stream=None):
        """From any object with n, off, col, directed (e.g. the inputs module's Graph)."""
        return cls(g.n, g.off, g.col, g.directed, stream)

    def set_param(self, param: int, value: float):
        """Tuning default for jobs created later on this graph (results do not change)."""
        _check(_lib.cen_graph_set_param(self.h, int(param), float(value)), "cen_graph_set_param")

    def close(self):
        if getattr(self, "h", None):
            _lib.cen_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Job:
    """The growing sample of one CentRA run (``cen_job_*``)."""

    def __init__(self, graph: Graph, seed: int, t: int, stream=None, space: int = 0, kappa: int = 0):
        self.graph = graph
        self.seed = int(seed)
        self.t = int(t)
        self.nw = (self.t + 31) // 32
        self.stream = stream if stream is not None else graph.stream
        h = ctypes.c_void_p()
        _check(_lib.cen_job_create_space(graph.h, self.seed, self.t, int(space), int(kappa), self.stream,
                                         ctypes.byref(h)), "cen_job_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.cen_job_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self):
        m, mem = ctypes.c_uint64(), ctypes.c_int64()
        _check(_lib.cen_job_size(self.h, ctypes.byref(m), ctypes.byref(mem)), "cen_job_size")
        return m.value, mem.value

    @property
    def m(self) -> int:
        return self.size()[0]

    def sample(self, m_new: int):
        _check(_lib.cen_sample(self.h, int(m_new)), "cen_sample")

    def greedy_cover(self, k: int):
        S = np.empty(k, np.int32)
        size, cov = ctypes.c_int32(), ctypes.c_uint64()
        _check(_lib.cen_greedy_cover(self.h, k, _p(S), ctypes.byref(size), ctypes.byref(cov)), "cen_greedy_cover")
        return S[: size.value].copy(), cov.value

    def mcera(self, k: int):
        Rnum = np.empty(self.t, np.int64)
        W, b = ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.cen_mcera(self.h, k, _p(Rnum), ctypes.byref(W), ctypes.byref(b)), "cen_mcera")
        return Rnum, W.value, b.value

    def cover_and_mcera(self, k: int):
        """``cen_cover_and_mcera``: greedy_cover(k) and mcera(k) side by side on two streams;
        returns (S, covered, Rnum, Wnum, b)."""
        S = np.empty(k, np.int32)
        size, cov = ctypes.c_int32(), ctypes.c_uint64()
        Rnum = np.empty(self.t, np.int64)
        W, b = ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.cen_cover_and_mcera(self.h, k, _p(S), ctypes.byref(size), ctypes.byref(cov), _p(Rnum),
                                        ctypes.byref(W), ctypes.byref(b)), "cen_cover_and_mcera")
        return S[: size.value].copy(), cov.value, Rnum, W.value, b.value

    def samples(self):
        m, mem = self.size()
        hoff = np.empty(m + 1, np.int64)
        hmem = np.empty(max(mem, 1), np.int32)
        s, t, d = (np.empty(max(m, 1), np.int32) for _ in range(3))
        _check(_lib.cen_job_copy_samples(self.h, _p(hoff), _p(hmem), _p(s), _p(t), _p(d)), "cen_job_copy_samples")
        return dict(hoff=hoff, hmem=hmem[:mem], s=s[:m], t=t[:m], d=d[:m])

    def incidence(self):
        _, mem = self.size()
        noff = np.empty(self.graph.n + 1, np.int64)
        nsamp = np.empty(max(mem, 1), np.int32)
        _check(_lib.cen_job_copy_incidence(self.h, _p(noff), _p(nsamp)), "cen_job_copy_incidence")
        return noff, nsamp[:mem]

    def rade(self):
        R = np.empty((self.t, self.graph.n), np.int32)
        c = np.empty(self.graph.n, np.int32)
        _check(_lib.cen_job_copy_rade(self.h, _p(R), _p(c)), "cen_job_copy_rade")
        return R, c

    def signs(self):
        m = self.m
        w = np.empty((max(m, 1), self.nw), np.uint32)
        _check(_lib.cen_job_copy_signs(self.h, _p(w)), "cen_job_copy_signs")
        return w[:m]

    def set_param(self, param: int, value: float):
        _check(_lib.cen_job_set_param(self.h, int(param), float(value)), "cen_job_set_param")

    # ---- one shard of a sample split over several GPUs (device buffers are torch CUDA tensors)
    def set_ids(self, stride: int, offset: int):
        """``cen_job_set_ids``: store position p holds sample id p * stride + offset."""
        _check(_lib.cen_job_set_ids(self.h, int(stride), int(offset)), "cen_job_set_ids")

    def shard_greedy_begin(self):
        _check(_lib.cen_shard_greedy_begin(self.h), "cen_shard_greedy_begin")

    def shard_gains(self, out):
        """This shard's gains into the int32 device tensor `out` [n]."""
        _check(_lib.cen_shard_gains(self.h, ctypes.c_void_p(out.data_ptr())), "cen_shard_gains")

    def shard_pick(self, gains):
        """(u, gain) of the summed gains `gains` (int32 device tensor [n]); u = -1 when all are 0."""
        u, g = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.cen_shard_pick(self.h, ctypes.c_void_p(gains.data_ptr()), ctypes.byref(u), ctypes.byref(g)),
               "cen_shard_pick")
        return u.value, g.value

    def shard_apply(self, u: int) -> int:
        newly = ctypes.c_uint64()
        _check(_lib.cen_shard_apply(self.h, int(u), ctypes.byref(newly)), "cen_shard_apply")
        return newly.value

    def shard_rade(self, out) -> int:
        """R (rows 0 .. t-1) and c (row t) of this shard into the int32 device tensor `out` [t+1][n]; returns b_H."""
        b = ctypes.c_int32()
        _check(_lib.cen_shard_rade(self.h, ctypes.c_void_p(out.data_ptr()), ctypes.byref(b)), "cen_shard_rade")
        return b.value

    def shard_topk(self, vals, nrows: int, k: int) -> np.ndarray:
        out = np.zeros(nrows, np.int64)
        _check(_lib.cen_shard_topk(self.h, ctypes.c_void_p(vals.data_ptr()), int(nrows), int(k), _p(out)),
               "cen_shard_topk")
        return out

    def tune(self, wave_words=None, wave_streams=None, push_ratio=None, level_budget=None, sampler=None,
             bidir_budget=None, bidir_queue=None, bidir_table=None, bidir_warps=None):
        """Speed and memory parameters (the samples do not depend on them)."""
        for p, v in ((PARAM_WAVE_WORDS, wave_words), (PARAM_WAVE_STREAMS, wave_streams),
                     (PARAM_PUSH_RATIO, push_ratio), (PARAM_LEVEL_BUDGET, level_budget), (PARAM_SAMPLER, sampler),
                     (PARAM_BIDIR_BUDGET, bidir_budget), (PARAM_BIDIR_QUEUE, bidir_queue),
                     (PARAM_BIDIR_TABLE, bidir_table), (PARAM_BIDIR_WARPS, bidir_warps)):
            if v is not None:
                self.set_param(p, v)

    def set_timing(self, enable: bool):
        _check(_lib.cen_job_set_timing(self.h, int(enable)), "cen_job_set_timing")

    def reset_stats(self):
        _check(_lib.cen_job_reset_stats(self.h), "cen_job_reset_stats")

    def sampler_info(self) -> dict:
        """``cen_job_sampler_info``: deferred_search, deferred_walk, migrated, slots, escalated."""
        a, b, m, c, e = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_uint64()
        _check(_lib.cen_job_sampler_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m), ctypes.byref(c),
                                         ctypes.byref(e)), "cen_job_sampler_info")
        return dict(deferred_search=a.value, deferred_walk=b.value, migrated=m.value, slots=c.value,
                    escalated=e.value)

    def stats(self) -> dict:
        arr = (cen_kstat * NKCLASS)()
        nc = ctypes.c_int32()
        _check(_lib.cen_job_stats(self.h, arr, ctypes.byref(nc)), "cen_job_stats")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, timed=arr[i].timed,
                                           units=arr[i].units) for i in range(nc.value)}


def release_cached():
    """``cen_release_cached``: frees device memory kept for reuse after jobs end."""
    _check(_lib.cen_release_cached(), "cen_release_cached")


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_installed = []  # callbacks the library may still call back (buffers go back to the allocator that made them)


def use_torch_allocator(enable: bool = True):
    """``cen_set_allocator``: take the library's device buffers from PyTorch's caching allocator (so
    ``torch.cuda.memory_allocated`` counts them and the two share one pool), or, with enable=False,
    from the stream-ordered device pool again.  Install it before creating graphs and jobs."""
    if not enable:
        _check(_lib.cen_set_allocator(None, None, None), "cen_set_allocator")
        return
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:  # out of memory: the library reports CEN_ENOMEM
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    fns = (_ALLOC_FN(alloc), _FREE_FN(free))
    _installed.append(fns)
    _check(_lib.cen_set_allocator(ctypes.cast(fns[0], ctypes.c_void_p), ctypes.cast(fns[1], ctypes.c_void_p), None),
           "cen_set_allocator")


def bounds(covered, m, Rsum, t, Wnum, b, eps, delta, i):
    """``cen_bounds``: (stop, dict C, A, w, nu, xi, Rt, R, eta)."""
    out = np.zeros(8, np.float64)
    stop = ctypes.c_int32()
    _check(_lib.cen_bounds(covered, m, Rsum, t, Wnum, b, eps, delta, i, _p(out), ctypes.byref(stop)), "cen_bounds")
    return bool(stop.value), dict(zip(("C", "A", "w", "nu", "xi", "Rt", "R", "eta"), out.tolist()))


def bounds_hedge(covered, m, n, k, eps, delta, i):
    """``cen_bounds_hedge``: (stop, dict C, LU, nuU, etaU) of HEDGE-P's union bound."""
    out = np.zeros(4, np.float64)
    stop = ctypes.c_int32()
    _check(_lib.cen_bounds_hedge(covered, m, n, k, eps, delta, i, _p(out), ctypes.byref(stop)), "cen_bounds_hedge")
    return bool(stop.value), dict(zip(("C", "LU", "nuU", "etaU"), out.tolist()))


def run(graph: Graph, k: int, eps: float, delta: float, t: int, seed: int, m0: int = 1000, m_cap: int = 1 << 30,
        stream=None, max_rounds: int = 64, schedule: int = 0, alpha: float = 1.2, rule: int = 0, space: int = 0,
        kappa: int = 0) -> dict:
    """``cen_run_ex`` (Algorithm 1): certified top-k set; status OK or ENOTCERTIFIED.
    schedule: SCHEDULE_DOUBLING (m0 2^(i-1)), SCHEDULE_PAPER (growth by alpha plus the optimistic guess) or
    SCHEDULE_EXTRAPOLATE (PAPER plus the last SD bound scaled to the stopping threshold);
    rule: RULE_CENTRA (AMCERA bounds) or RULE_HEDGE_P (union bound); space: SPACE_* (kappa for SPACE_KPATH)."""
    S = np.empty(k, np.int32)
    size, rounds = ctypes.c_int32(), ctypes.c_int32()
    cov, mf = ctypes.c_uint64(), ctypes.c_uint64()
    log = np.zeros((max_rounds, 16), np.float64)
    st = stream if stream is not None else graph.stream
    opts = cen_run_opts(schedule, rule, alpha, space, kappa)
    rc = _lib.cen_run_ex(graph.h, k, eps, delta, t, seed, m0, m_cap, ctypes.byref(opts), st, _p(S),
                         ctypes.byref(size), ctypes.byref(cov), ctypes.byref(mf), ctypes.byref(rounds), _p(log),
                         max_rounds)
    if rc not in (OK, ENOTCERTIFIED):
        _check(rc, "cen_run")
    return dict(status=rc, S=S[: size.value].copy(), covered=cov.value, m_final=mf.value, rounds=rounds.value,
                log=log[: min(rounds.value, max_rounds)].copy())


def run_batch(jobs, nworkers: int = 8, max_rounds: int = 64) -> list[dict]:
    """``cen_run_batch``: `jobs` is a list of dicts with graph (Graph), k, eps, delta, t, seed and optional
    m0 (1000) / m_cap (2^30) / schedule (0) / rule (0) / alpha (1.2) / space (0) / kappa (0).  Returns one dict per job, like ``run`` plus start_s / end_s."""
    n = len(jobs)
    specs = (cen_job_spec * max(n, 1))()
    res = (cen_job_result * max(n, 1))()
    keep = []
    for i, j in enumerate(jobs):
        specs[i] = cen_job_spec(j["graph"].h, j["k"], j["t"], j["eps"], j["delta"], j["seed"], j.get("m0", 1000),
                                j.get("m_cap", 1 << 30),
                                cen_run_opts(j.get("schedule", 0), j.get("rule", 0), j.get("alpha", 1.2),
                                             j.get("space", 0), j.get("kappa", 0)))
        S = np.empty(j["k"], np.int32)
        log = np.zeros((max_rounds, 16), np.float64)
        keep.append((S, log))
        res[i].S = S.ctypes.data
        res[i].log = log.ctypes.data
        res[i].max_rounds = max_rounds
    _check(_lib.cen_run_batch(specs, n, nworkers, res), "cen_run_batch")
    out = []
    for i in range(n):
        S, log = keep[i]
        r = res[i]
        out.append(dict(status=r.status, S=S[: r.S_size].copy(), covered=r.covered, m_final=r.m_final,
                        rounds=r.rounds, log=log[: min(r.rounds, max_rounds)].copy(), start_s=r.start_s,
                        end_s=r.end_s))
    return out


def run_result(job: dict, stream=None, max_rounds: int = 64) -> dict:
    """``cen_run_result``: one run from a spec dict (as for ``run_batch``) into the result struct;
    returns dict(status, S, covered, m_final, rounds, log, seconds)."""
    g = job["graph"]
    spec = cen_job_spec(g.h, job["k"], job["t"], job["eps"], job["delta"], job["seed"], job.get("m0", 1000),
                        job.get("m_cap", 1 << 30),
                        cen_run_opts(job.get("schedule", 0), job.get("rule", 0), job.get("alpha", 1.2),
                                     job.get("space", 0), job.get("kappa", 0)))
    S = np.empty(job["k"], np.int32)
    log = np.zeros((max_rounds, 16), np.float64)
    res = cen_job_result()
    res.S = S.ctypes.data
    res.log = log.ctypes.data
    res.max_rounds = max_rounds
    rc = _lib.cen_run_result(ctypes.byref(spec), stream if stream is not None else g.stream, ctypes.byref(res))
    if rc not in (OK, ENOTCERTIFIED):
        _check(rc, "cen_run_result")
    return dict(status=rc, S=S[: res.S_size].copy(), covered=res.covered, m_final=res.m_final, rounds=res.rounds,
                log=log[: min(res.rounds, max_rounds)].copy(), seconds=res.end_s)
