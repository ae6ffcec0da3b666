"""Host-side helpers of bench.py: the DRAM view of the roofline and the
reading of a committed ncu summary (valid only for the kernel source it was
taken on)."""
import pytest

import bench


def test_dram_view_from_recorded_profile():
    v = bench.dram_view({"dram_bytes_per_launch_full_workload": 1e9, "l2_sector_hit_pct": 90.0}, 100.0, 5000.0)
    assert v["gbs"] == pytest.approx(10.0)
    assert v["frac"] == pytest.approx(0.002)
    assert v["l2_sector_hit_pct"] == 90.0 and v["l1_sector_hit_pct"] is None
    assert bench.dram_view({}, 100.0, 5000.0) is None


def test_pipe_view_needs_every_figure():
    prof = {"issue_active_pct": 74.0, "alu_pipe_pct": 61.0, "fma_pipe_pct": 22.0, "thread_inst_per_segment": 99.0}
    v = bench.pipe_view(prof)
    assert v["alu_pipe_pct"] == 61.0 and "source" in v
    assert bench.pipe_view({"issue_active_pct": 74.0}) is None


def test_recorded_profile_requires_matching_kernel_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "batch_kernel_demo_traffic.txt").write_text(
        "# comment: ignored\nkernel_source_sha: abc123\ndram_bytes_per_launch_full_workload: 4096\n"
        "l1_sector_hit_pct: 80.5\nl2_sector_hit_pct: not-a-number\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    assert bench.recorded_profile("demo") == {"dram_bytes_per_launch_full_workload": 4096.0, "l1_sector_hit_pct": 80.5}
    assert bench.recorded_traffic("demo") == 4096.0
    assert bench.recorded_profile("missing") == {}
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.recorded_profile("demo") == {} and bench.recorded_traffic("demo") is None
