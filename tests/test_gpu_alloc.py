"""Device memory from a caller's allocator (cen_set_allocator): with PyTorch's
caching allocator installed, the library's buffers show up in
torch.cuda.memory_allocated, all of them go back when the graph and job are
freed, and the results are the same as with the stream-ordered pool."""
import numpy as np
import pytest

import oracle as O
from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2306_03651_gb300")


def run_once(g, stream=None):
    graph = P.Graph.of(g, stream=stream)
    job = P.Job(graph, 5, 16)
    job.sample(3000)
    job.sample(5000)  # grows the sample store: buffers are reallocated and freed
    S, covered = job.greedy_cover(10)
    Rn, Wn, b = job.mcera(10)
    samples = job.samples()
    job.close()
    graph.close()
    return S, covered, Rn, Wn, b, samples


def test_torch_allocator_owns_and_returns_everything():
    torch = pytest.importorskip("torch")
    g = I.ba(2000, 4, 1)
    ref = run_once(g)
    P.release_cached()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    P.use_torch_allocator()
    try:
        graph = P.Graph.of(g)
        job = P.Job(graph, 5, 16)
        job.sample(3000)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() > base  # the graph, samples and workspaces came from torch
        job.close()
        graph.close()
        got = run_once(g, stream=P.current_stream())
        P.release_cached()  # cached sampler workspaces go back too
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        P.use_torch_allocator(False)
        P.release_cached()
        torch.cuda.empty_cache()
    assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
    assert np.array_equal(got[2], ref[2]) and got[3:5] == ref[3:5]
    for key in ("hoff", "s", "t", "d", "hmem"):
        assert np.array_equal(got[5][key], ref[5][key]), key
    # and both agree with the oracle
    oj = O.Job(O.Graph.of(g), 5, 16)
    oj.sample(3000)
    oj.sample(5000)
    assert np.array_equal(oj.hypergraph()["hmem"], got[5]["hmem"])


def test_set_allocator_needs_both_functions():
    P.cen_set_allocator(None, None, None)
    rc = P.cen_set_allocator(P._ALLOC_FN(lambda n, s, c: None), None, None)
    assert rc == P.EINVAL
