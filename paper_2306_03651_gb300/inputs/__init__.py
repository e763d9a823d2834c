"""Seeded synthetic graphs shaped like the paper's workloads (Sec. 5, Table 1).

This module is input plumbing only: it holds none of the sampling, covering or
bounding arithmetic, imports nothing else from the package, and serves both the
CUDA path and the CPU oracle with identical CSR arrays.

Every graph is returned as a canonical CSR (rows ascending, no duplicate arcs,
no self-loops; undirected graphs hold both arcs of each edge):
``Graph(n, off: int64[n+1], col: int32[nnz], directed: bool, name: str)``.

The paper's SNAP/KONECT graphs are not available offline; the stand-ins are
  * Barabasi-Albert preferential attachment (small-world, hubs),
  * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with (a,b,c,d) = (.57,.19,.19,.05),
  * a 4-neighbour grid with 1% of its edges rewired (the high-diameter regime).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libcengen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C generators into ``libcengen.so`` next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32, i64, u64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.gen_ba.argtypes = [i32, i32, u64, vp, pp]
        lib.gen_ba.restype = i64
        lib.gen_rmat_edges.argtypes = [i32, i64, dbl, dbl, dbl, u64, vp, vp]
        lib.gen_rmat_edges.restype = None
        lib.gen_csr_from_edges.argtypes = [i32, i64, vp, vp, ctypes.c_int, vp, pp]
        lib.gen_csr_from_edges.restype = i64
        lib.gen_lcc.argtypes = [i32, vp, vp, vp]
        lib.gen_lcc.restype = i32
        lib.gen_induce.argtypes = [i32, vp, vp, vp, i32, vp, pp]
        lib.gen_induce.restype = i64
        lib.gen_grid_rewired.argtypes = [i32, i32, dbl, u64, vp, pp]
        lib.gen_grid_rewired.restype = i64
        lib.gen_draw_u64.argtypes = [u64, i64, vp]
        lib.gen_draw_u64.restype = None
        lib.gen_free.argtypes = [vp]
        lib.gen_free.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _take_col(lib, cptr: ctypes.c_void_p, nnz: int) -> np.ndarray:
    buf = (ctypes.c_int32 * max(nnz, 1)).from_address(cptr.value)
    col = np.frombuffer(buf, dtype=np.int32, count=nnz).copy()
    lib.gen_free(cptr)
    return col


@dataclass
class Graph:
    n: int
    off: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    directed: bool
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def from_edges(n: int, src, dst, directed: bool, name: str = "") -> Graph:
    """Canonical CSR from an arc list (both arcs are added when undirected)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    off = np.zeros(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    nnz = lib.gen_csr_from_edges(n, len(src), _ptr(src), _ptr(dst), 0 if directed else 1, _ptr(off),
                                 ctypes.byref(cptr))
    return Graph(n, off, _take_col(lib, cptr, nnz), directed, name)


def ba(n: int, d: int, seed: int) -> Graph:
    """Barabasi-Albert: K_{d+1} seed graph, then d distinct degree-proportional targets per new node."""
    lib = _load()
    off = np.zeros(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    nnz = lib.gen_ba(n, d, seed, _ptr(off), ctypes.byref(cptr))
    if nnz < 0:
        raise ValueError("ba: need d >= 1 and n >= d + 1")
    return Graph(n, off, _take_col(lib, cptr, nnz), False, f"ba(n={n},d={d},seed={seed})")


def rmat_edges(scale: int, edge_factor: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 1):
    lib = _load()
    ne = edge_factor << scale
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    a, b, c, _ = abcd
    lib.gen_rmat_edges(scale, ne, a, b, c, seed, _ptr(src), _ptr(dst))
    return src, dst


def lcc(g: Graph) -> Graph:
    """Largest connected component of an undirected graph, ids relabelled in original order."""
    lib = _load()
    keep = np.empty(g.n, dtype=np.int32)
    n_new = lib.gen_lcc(g.n, _ptr(g.off), _ptr(g.col), _ptr(keep))
    off = np.zeros(n_new + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    nnz = lib.gen_induce(g.n, _ptr(g.off), _ptr(g.col), _ptr(keep), n_new, _ptr(off), ctypes.byref(cptr))
    return Graph(n_new, off, _take_col(lib, cptr, nnz), False, g.name + "+lcc")


def rmat(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 1, directed: bool = False,
         keep_lcc: bool = True) -> Graph:
    src, dst = rmat_edges(scale, edge_factor, abcd, seed)
    g = from_edges(1 << scale, src, dst, directed, f"rmat(scale={scale},ef={edge_factor},seed={seed},"
                                                     f"{'directed' if directed else 'undirected'})")
    if not directed and keep_lcc:
        g = lcc(g)
    return g


def grid_rewired(width: int, height: int, p: float = 0.01, seed: int = 1) -> Graph:
    lib = _load()
    n = width * height
    off = np.zeros(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    nnz = lib.gen_grid_rewired(width, height, p, seed, _ptr(off), ctypes.byref(cptr))
    return Graph(n, off, _take_col(lib, cptr, nnz), False, f"grid({width}x{height},p={p},seed={seed})")


def draw_u64(seed: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.gen_draw_u64(seed, count, _ptr(out))
    return out


# ------------------------------------------------------------------ workloads
@dataclass
class Workload:
    """One CentRA problem instance: a graph plus the method's parameters."""
    graph: Graph
    k: int
    eps: float
    delta: float
    t: int
    seed: int
    m0: int = 1000


def ba_2000() -> Workload:
    """BA n=2,000, 4 edges per new node (~8k edges), graph seed 1; k=10, eps=0.05, delta=0.1, t=10."""
    return Workload(ba(2000, 4, 1), k=10, eps=0.05, delta=0.1, t=10, seed=1)


def rmat18_lcc() -> Workload:
    """Undirected R-MAT scale 18, edge factor 16, LCC; k=50, eps=0.01, delta=0.1, t=10."""
    return Workload(rmat(18, 16, seed=1, directed=False, keep_lcc=True), k=50, eps=0.01, delta=0.1, t=10, seed=1)


def grid2048_rewired() -> Workload:
    """2048x2048 4-neighbour grid, 1% of edges rewired; k=100, eps=0.005, delta=0.05, t=100."""
    return Workload(grid_rewired(2048, 2048, 0.01, seed=1), k=100, eps=0.005, delta=0.05, t=100, seed=1)


def rmat22_directed() -> Workload:
    """Directed R-MAT scale 22, edge factor 16 (no LCC); k=100, eps=0.005, delta=0.05, t=100."""
    return Workload(rmat(22, 16, seed=1, directed=True, keep_lcc=False), k=100, eps=0.005, delta=0.05, t=100,
                    seed=1)


def ba_batch_params(njobs: int = 64, seed: int = 7):
    """Parameters of the batched workload: n log-uniform in [1e4, 5e5], d in {2..8}, k in {10, 50, 100}."""
    r = draw_u64(seed, 3 * njobs)
    out = []
    for j in range(njobs):
        u = float(r[3 * j] >> np.uint64(11)) / float(1 << 53)
        n = int(round(math.exp(math.log(1e4) + u * (math.log(5e5) - math.log(1e4)))))
        d = 2 + int(r[3 * j + 1] % np.uint64(7))
        k = (10, 50, 100)[int(r[3 * j + 2] % np.uint64(3))]
        out.append(dict(n=n, d=d, k=k, graph_seed=1000 + j, job_seed=j))
    return out


def ba_batch(njobs: int = 64, eps: float = 0.01, delta: float = 0.1, t: int = 32, scale: float = 1.0):
    """The batched workload: `njobs` BA graphs (n scaled by `scale` for small test variants)."""
    jobs = []
    for p in ba_batch_params(njobs):
        n = max(p["d"] + 2, int(p["n"] * scale))
        jobs.append(Workload(ba(n, p["d"], p["graph_seed"]), k=p["k"], eps=eps, delta=delta, t=t, seed=p["job_seed"]))
    return jobs
