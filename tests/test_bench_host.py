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
