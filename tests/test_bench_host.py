"""Host-side logic of bench.py and of the serving loop (no GPU): the DRAM-traffic lookup is
reported only while the profiled source is unchanged; the clock sampler reads a window of
samples; the admission estimate counts the bidirectional workspace and grows with the sample
cap; and admission is FIFO within the worker count and the byte budget."""
import hashlib
import os

import pytest

import bench
from paper_2306_03651_gb300 import serve


def test_dram_traffic_is_guarded_by_the_source_hash_and_workload(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    (prof_dir / "k_dram.md").write_text(f"# t\n\ntraffic_bytes_per_launch: 1234\nkernel_class: k\n"
                                          f"workload: w\npairs_per_step: 64\nsource_sha256_16: {sha}\n")
    csrc = tmp_path / "paper_2306_03651_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "kernel.cu").write_bytes(src.read_bytes())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "DRAM_PROFILES", {"k": ("k_dram.md", "kernel.cu")})
    assert bench.dram_traffic("k", "w", 64) == 1234.0
    assert bench.dram_traffic("other", "w", 64) is None
    assert bench.dram_traffic("k", "w2", 64) is None  # another workload's launch
    assert bench.dram_traffic("k", "w", 128) is None  # another step size
    (csrc / "kernel.cu").write_text("// changed\n")
    assert bench.dram_traffic("k", "w", 64) is None


def test_committed_profiles_name_their_class_and_source():
    for cls, (prof, src) in bench.DRAM_PROFILES.items():
        text = open(os.path.join(bench.ROOT, "profiles", prof)).read()
        assert f"kernel_class: {cls}" in text and "source_sha256_16:" in text and "traffic_bytes_per_launch:" in text
        assert "workload:" in text and "pairs_per_step:" in text
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2306_03651_gb300", "csrc", src))


def test_serving_estimate_counts_the_sampler_workspace():
    small = serve.estimate_job_bytes(2000, 16000, 10, 1 << 20)
    big_cap = serve.estimate_job_bytes(2000, 16000, 10, 1 << 24)
    assert big_cap > small
    n = 1 << 20  # large enough that the default budget, not the CTA count, sets the workspace
    roomy = serve.estimate_job_bytes(n, 16 * n, 10, 1 << 20)
    tight = serve.estimate_job_bytes(n, 16 * n, 10, 1 << 20, bidir_budget=1 << 28)
    assert roomy - tight > (1 << 30)
    with pytest.raises(TypeError):
        serve.estimate_job_bytes(2000)


def test_clock_sampler_reads_a_window_of_samples(tmp_path, monkeypatch):
    # a stand-in nvidia-smi: 1,500 MHz for its first lines, then 2,070 MHz with power capping
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "for i in 1 2 3; do echo '0, 1500, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active';"
                    " sleep 0.02; done\n"
                    "while true; do echo '0, 2070, 2070, 900, 0x4, Not Active, Not Active, Not Active, Active';"
                    " sleep 0.02; done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    import time
    c = bench.ClockSampler(0)
    c.start()
    assert c.lines  # start() returns once sampling runs
    time.sleep(0.15)
    t0 = time.perf_counter()
    time.sleep(0.15)
    t1 = time.perf_counter()
    time.sleep(0.05)
    r = c.stop(t0, t1)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] >= 3
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.05)
    r = c.stop()  # no window: every sample counts, the early 1,500 MHz ones too
    assert r["samples"] >= 2 and r["sm_max_mhz"] == 2070.0


class _FakeStream:
    cuda_stream = 0


class _FakeGraph:
    def __init__(self, n, nnz):
        self.n, self.nnz = n, nnz


def test_server_admission_by_budget_and_fifo(monkeypatch):
    """The serving loop's host logic with a stand-in runner: requests start in arrival
    order, never more at once than the workers or the byte budget allow, and every request
    finishes with its own result."""
    import threading
    import time
    import numpy as np
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _FakeStream())
    running, peak, started = [0], [0], []
    lock = threading.Lock()

    def fake_runner(g, req, stream, reserve):
        reserve(req.m0)
        with lock:
            running[0] += 1
            peak[0] = max(peak[0], running[0])
            started.append(req.seed)
        time.sleep(0.03)
        with lock:
            running[0] -= 1
        return {"status": serve.P.OK, "S": np.arange(req.k, dtype=np.int32), "covered": req.seed, "m_final": 1000,
                "rounds": 1, "log": np.zeros((1, 16))}

    graphs = {"a": _FakeGraph(2000, 16000)}
    per_job = serve.estimate_job_bytes(2000, 16000, 8, 1000)
    reqs = [serve.Request(rid=i, graph="a", k=5, eps=0.1, delta=0.1, t=8, seed=100 + i, arrival_s=0.002 * i,
                          m_cap=1 << 20) for i in range(12)]
    # budget for two jobs at a time, four workers
    srv = serve.Server(graphs, workers=4, hbm_budget_bytes=2 * per_job, runner=fake_runner)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(12))
    assert all(r.covered == 100 + r.rid and r.status == serve.P.OK for r in res)
    st = [r.start_s for r in res]  # FIFO: admitted in arrival order (thread start may jitter by a few ms)
    assert all(a <= b + 0.01 for a, b in zip(st, st[1:]))
    assert peak[0] <= 2 and srv.peak_running <= 2 and srv.peak_bytes <= 2 * per_job
    # budget for all, two workers: the workers bound it
    running[0], peak[0] = 0, 0
    started.clear()
    srv = serve.Server(graphs, workers=2, hbm_budget_bytes=100 * per_job, runner=fake_runner)
    res2 = srv.serve(reqs)
    st = [r.start_s for r in res2]
    assert peak[0] <= 2 and all(a <= b + 0.01 for a, b in zip(st, st[1:]))
    summ = serve.summarize(res)
    assert summ["jobs"] == 12 and summ["certified"] == 12


def test_server_growth_reservations_wait_and_never_deadlock(monkeypatch):
    """Requests reserve the memory of each grown round: with room for three first rounds
    but not for all of their growth, rounds wait for older requests to finish, and every
    request finishes.  Only the oldest running request grows without waiting, so the
    total stays within the budget plus one request's growth."""
    import time
    import numpy as np
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _FakeStream())
    graphs = {"a": _FakeGraph(20000, 160000)}
    m0, rounds = 1 << 16, 4
    est = [serve.estimate_job_bytes(20000, 160000, 8, m0 << r) for r in range(rounds)]
    budget = est[rounds - 1] + 2 * est[0]  # one request at its largest round and two first rounds

    def fake_runner(g, req, stream, reserve):
        for r in range(rounds):
            reserve(m0 << r)
            time.sleep(0.01)
        return {"status": serve.P.OK, "S": np.zeros(0, np.int32), "covered": 0, "m_final": m0 << (rounds - 1),
                "rounds": rounds, "log": np.zeros((rounds, 16))}

    reqs = [serve.Request(rid=i, graph="a", k=5, eps=0.1, delta=0.1, t=8, seed=i, m0=m0, m_cap=1 << 30)
            for i in range(8)]
    srv = serve.Server(graphs, workers=4, hbm_budget_bytes=budget, runner=fake_runner)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(8)) and all(r.status == serve.P.OK for r in res)
    assert srv.peak_bytes <= budget + est[rounds - 1] - est[0] and srv.peak_running >= 2 and srv.waits > 0
    assert srv._in_use == 0


def test_server_failed_request_gets_a_result_and_frees_its_slot(monkeypatch):
    """A run that raises (e.g. ENOMEM when the byte estimate was too low) ends that request
    with its error status and message, and gives its worker and its bytes back: with one
    worker, the requests after it still run."""
    import numpy as np
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _FakeStream())

    def fake_runner(g, req, stream, reserve):
        reserve(req.m0)
        if req.seed % 3 == 0:
            raise serve.P.CenError(serve.P.ENOMEM, "out of device memory")
        return {"status": serve.P.OK, "S": np.arange(req.k, dtype=np.int32), "covered": req.seed, "m_final": 1000,
                "rounds": 1, "log": np.zeros((1, 16))}

    graphs = {"a": _FakeGraph(2000, 16000)}
    per_job = serve.estimate_job_bytes(2000, 16000, 8, 1000)
    reqs = [serve.Request(rid=i, graph="a", k=5, eps=0.1, delta=0.1, t=8, seed=i, m_cap=1 << 20) for i in range(7)]
    srv = serve.Server(graphs, workers=1, hbm_budget_bytes=per_job, runner=fake_runner)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(7))
    for r in res:
        if r.rid % 3 == 0:
            assert r.status == serve.P.ENOMEM and "out of device memory" in r.error and len(r.S) == 0
        else:
            assert r.status == serve.P.OK and r.covered == r.rid and r.error == ""
    assert srv._in_use == 0 and srv._free_workers == [0]
    assert serve.summarize(res)["certified"] == 4
