"""Host-side logic of bench.py and the serving estimate (no GPU): the DRAM-traffic lookup is
reported only while the profiled source is unchanged, and the admission estimate counts the
bidirectional workspace and grows with the sample cap."""
import hashlib
import os

import pytest

import bench
from paper_2306_03651_gb300 import serve


def test_dram_traffic_is_guarded_by_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    (prof_dir / "k_dram.md").write_text(f"# t\n\ntraffic_bytes_per_launch: 1234\nkernel_class: k\nsource_sha256_16: {sha}\n")
    csrc = tmp_path / "paper_2306_03651_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "kernel.cu").write_bytes(src.read_bytes())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "DRAM_PROFILES", {"k": ("k_dram.md", "kernel.cu")})
    assert bench.dram_traffic("k") == 1234.0
    assert bench.dram_traffic("other") is None
    (csrc / "kernel.cu").write_text("// changed\n")
    assert bench.dram_traffic("k") is None


def test_committed_profiles_name_their_class_and_source():
    for cls, (prof, src) in bench.DRAM_PROFILES.items():
        text = open(os.path.join(bench.ROOT, "profiles", prof)).read()
        assert f"kernel_class: {cls}" in text and "source_sha256_16:" in text and "traffic_bytes_per_launch:" in text
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
