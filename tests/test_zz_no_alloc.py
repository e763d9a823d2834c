"""The allocation-free entry point against cen_mcera.

cen_topk_positive_sum_noalloc serves callers that cannot allocate device
memory (another runtime or pool owns the device, or a host callback in which
cudaMalloc/cudaFree are not allowed); its scratch is a static device array.
Here its output must equal what cen_mcera reports for the same job -- the
per-vector sums Rnum over the job's R matrix and Wnum over its c vector --
on two calls in a row, which also checks that leftovers in the shared array
from the first call do not leak into the second.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_2306_03651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def noalloc(P, torch, mat: np.ndarray, k: int) -> np.ndarray:
    mat = np.ascontiguousarray(mat, dtype=np.int32)
    nrows, n = mat.shape
    dev = torch.from_numpy(mat).cuda()  # the caller owns inputs and outputs
    torch.cuda.synchronize()
    out = np.full(nrows, -1, np.int64)
    rc = P.cen_topk_positive_sum_noalloc(ctypes.c_void_p(dev.data_ptr()), n, nrows, k, out.ctypes.data,
                                         P.current_stream())
    assert rc == P.OK, P.last_error()
    return out


def test_noalloc_matches_mcera_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_2306_03651_gb300 as P
    g = I.ba(3000, 3, 4)
    t = 40
    job = P.Job(P.Graph.of(g), 17, t)
    job.sample(5000)
    for k in (1, 7, 50, 5000):
        Rnum, Wnum, _ = job.mcera(k)
        R, c = job.rade()
        for _ in range(2):
            assert np.array_equal(noalloc(P, torch, R, k), Rnum)
            assert noalloc(P, torch, c[None, :], k)[0] == Wnum


def test_noalloc_rejects_too_many_rows():
    torch = pytest.importorskip("torch")
    import paper_2306_03651_gb300 as P
    mat = np.ones((129, 10), np.int32)
    dev = torch.from_numpy(mat).cuda()
    out = np.zeros(129, np.int64)
    rc = P.cen_topk_positive_sum_noalloc(ctypes.c_void_p(dev.data_ptr()), 10, 129, 3, out.ctypes.data,
                                         P.current_stream())
    assert rc == P.EINVAL and "128" in P.last_error()
