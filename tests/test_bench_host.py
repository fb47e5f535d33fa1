"""Host logic of bench.py on the CPU: the DRAM traffic of the roofline object
comes from the committed ncu summary only while the kernel's sources hash to
the value recorded with it (else null), and the summary in the repository
states both lines."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    a, b = tmp_path / "k.cu", tmp_path / "k.cuh"
    a.write_text("kernel A\n")
    b.write_text("header B\n")
    prof = tmp_path / "summary.md"
    prof.write_text(f"text\ntraffic_bytes_per_launch: 123456\nkernel_sources_sha256_16: "
                    f"{bench.sources_sha([str(a), str(b)])}\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profile_traffic([str(a), str(b)]) == 123456.0
    a.write_text("kernel A, changed\n")  # the kernel changed since the capture
    assert bench.profile_traffic([str(a), str(b)]) is None
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profile_traffic([str(a), str(b)]) is None


def test_committed_summary_states_traffic_and_hash():
    lines = open(bench.PROFILE).read().splitlines()
    traffic = [ln for ln in lines if ln.startswith("traffic_bytes_per_launch:")]
    sha = [ln for ln in lines if ln.startswith("kernel_sources_sha256_16:")]
    assert len(traffic) == 1 and float(traffic[0].split(":", 1)[1]) > 0
    assert len(sha) == 1 and len(sha[0].split(":", 1)[1].strip()) == 16
    assert all(os.path.exists(p) for p in bench.KERNEL_SOURCES)
