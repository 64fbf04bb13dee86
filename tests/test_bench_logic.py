"""Host logic of bench.py (no GPU): whole-job MLUPS, the roofline traffic
lookup (a committed ncu figure is used only while the kernel source is the
one it was taken from), and the measured peak with its fallback."""
import json
import os

import bench


def test_aggregate_mlups():
    # 2 ranks x 1000 nodes x 10 steps in 5 ms
    assert bench.aggregate_mlups(1000, 10, 5.0, 2) == 2 * 1000 * 10 / 5e-3 / 1e6


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (tmp_path / "paper_2005_08674_gb300").symlink_to(os.path.join(bench.ROOT, "paper_2005_08674_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_sha()
    (prof / "x_traffic_f32.md").write_text(f"kernel_source_sha: {sha}\ndram_bytes_per_cell: 70.5\n")
    assert bench.profiled_traffic("x_traffic", "f32", 1000) == 70.5 * 1000
    (prof / "x_traffic_f32.md").write_text("kernel_source_sha: 0123456789abcdef\ndram_bytes_per_cell: 70.5\n")
    assert bench.profiled_traffic("x_traffic", "f32", 1000) is None
    assert bench.profiled_traffic("missing", "f32", 1000) is None


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_gbs() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6784.2}))
    assert bench.measured_peak_gbs() == (6784.2, "measured")
