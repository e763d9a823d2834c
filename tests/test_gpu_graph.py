"""GPU graph loading (the graph G = (V, E) of Sec. 3.1): canonicalizing and
symmetrizing an arbitrary CSR on the device gives, array for array, the
canonical CSR the inputs module builds on the CPU from the same arc list."""
import numpy as np
import pytest

from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2306_03651_gb300")


def raw_csr(n, src, dst, seed):
    """CSR grouped by tail, rows in a shuffled order, repeats and self-loops kept."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(src))
    src, dst = np.asarray(src)[perm], np.asarray(dst)[perm]
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, np.asarray(src, np.int64) + 1, 1)
    return np.cumsum(off), np.asarray(dst, np.int32)[order]


def expected(n, src, dst, both):
    """The canonical rows by the plain definition: unique (u, v), u != v, sorted."""
    s, d = np.asarray(src, np.int64), np.asarray(dst, np.int64)
    if both:
        s, d = np.concatenate([s, d]), np.concatenate([d, s])
    keep = s != d
    key = np.unique(s[keep] * n + d[keep])
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, key // n + 1, 1)
    return np.cumsum(off), (key % n).astype(np.int32)


@pytest.mark.parametrize("scale,directed", [(10, False), (10, True), (14, False), (14, True)])
def test_canonicalize_rmat(scale, directed):
    src, dst = I.rmat_edges(scale, 8, seed=11)
    n = 1 << scale
    off, col = raw_csr(n, src, dst, scale)
    flags = P.GRAPH_CANONICALIZE | (0 if directed else P.GRAPH_SYMMETRIZE)
    g = P.Graph(n, off, col, directed, flags=flags)
    goff, gcol = g.csr()
    ref = I.from_edges(n, src, dst, directed)
    eoff, ecol = expected(n, src, dst, not directed)
    assert np.array_equal(ref.off, eoff) and np.array_equal(ref.col, ecol)  # the two CPU builders agree
    assert g.nnz == ref.nnz
    assert np.array_equal(goff, ref.off)
    assert np.array_equal(gcol, ref.col)


def test_canonicalize_device_input_and_run():
    torch = pytest.importorskip("torch")
    src, dst = I.rmat_edges(11, 8, seed=5)
    n = 1 << 11
    off, col = raw_csr(n, src, dst, 1)
    g = P.Graph(n, torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda(), False,
                flags=P.GRAPH_CANONICALIZE | P.GRAPH_SYMMETRIZE)
    ref = I.from_edges(n, src, dst, False)
    goff, gcol = g.csr()
    assert np.array_equal(goff, ref.off) and np.array_equal(gcol, ref.col)
    # the same graph gives the same run, whichever way it was loaded
    a = P.run(g, 10, 0.2, 0.1, 16, 3, m0=500)
    b = P.run(P.Graph.of(ref), 10, 0.2, 0.1, 16, 3, m0=500)
    assert a["status"] == b["status"] and np.array_equal(a["S"], b["S"]) and a["m_final"] == b["m_final"]


def test_canonical_input_unchanged_and_edge_cases():
    g0 = I.ba(500, 3, 2)
    g = P.Graph(g0.n, g0.off, g0.col, False, flags=P.GRAPH_CANONICALIZE)
    off, col = g.csr()
    assert np.array_equal(off, g0.off) and np.array_equal(col, g0.col)
    # only self-loops and repeats: nothing is kept
    n = 5
    g = P.Graph(n, np.array([0, 3, 3, 3, 3, 3]), np.array([0, 0, 0], np.int32), True, flags=P.GRAPH_CANONICALIZE)
    off, col = g.csr()
    assert g.nnz == 0 and not off.any()
    # one arc, symmetrized
    g = P.Graph(n, np.array([0, 0, 1, 1, 1, 1]), np.array([4], np.int32), False,
                flags=P.GRAPH_CANONICALIZE | P.GRAPH_SYMMETRIZE)
    off, col = g.csr()
    assert off.tolist() == [0, 0, 1, 1, 1, 2] and col.tolist() == [4, 1]


def test_canonicalize_rejects():
    n = 4
    with pytest.raises(RuntimeError, match="ids lie in"):  # id out of range
        P.Graph(n, np.array([0, 1, 1, 1, 1]), np.array([4], np.int32), True, flags=P.GRAPH_CANONICALIZE)
    with pytest.raises(RuntimeError, match="offsets"):  # offsets fall
        P.Graph(n, np.array([0, 2, 1, 2, 2]), np.array([1, 2], np.int32), True, flags=P.GRAPH_CANONICALIZE)
    with pytest.raises(RuntimeError, match="undirected"):
        P.Graph(n, np.array([0, 1, 1, 1, 1]), np.array([2], np.int32), True, flags=P.GRAPH_SYMMETRIZE)
    with pytest.raises(RuntimeError, match="not canonical"):  # without the flag a repeat is rejected
        P.Graph(n, np.array([0, 2, 2, 2, 2]), np.array([1, 1], np.int32), True)
