"""Host-side helpers of bench.py (no GPU): the roofline traffic is reported only for the kernel
sources it was measured on, and the measured peak is read from the driver's file when present."""
import json

import bench


def test_traffic_follows_the_recorded_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    assert bench.kernel_source_hash("large96") != h  # the 96^3 passes are built from other sources
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "pair_passes_w_traffic.txt").write_text(json.dumps(
        {"source_sha256_16": h, "dram_bytes_per_launch": {"5": 123}}))
    (prof / "pair_passes_old_traffic.txt").write_text(json.dumps(
        {"source_sha256_16": "0" * 16, "dram_bytes_per_launch": {"5": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda workload="default": h)
    assert bench.profiled_traffic(5, "w", True) == (123.0, "profiles/pair_passes_w_traffic.txt")
    assert bench.profiled_traffic(6, "w", True) == (None, None)
    assert bench.profiled_traffic(5, "w", False) == (None, None)
    assert bench.profiled_traffic(5, "old", True)[0] is None
    assert bench.profiled_traffic(5, "missing", True) == (None, None)


def test_measured_peak_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.6}))
    assert bench.measured_peaks() == (6789.6, "measured")


def test_traffic_is_scaled_to_another_block_size(tmp_path, monkeypatch):
    """A run with another pair block than the capture's gets the recorded traffic scaled by its
    orbitals, and says so."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "pair_passes_w_traffic.txt").write_text(json.dumps(
        {"source_sha256_16": "x" * 16, "dram_bytes_per_launch": {"5": 1000}, "algorithmic_bytes_per_launch": 800}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda workload="default": "x" * 16)
    assert bench.profiled_traffic(5, "w", True, 800) == (1000.0, "profiles/pair_passes_w_traffic.txt")
    v, note = bench.profiled_traffic(5, "w", True, 400)
    assert v == 500.0 and "scaled" in note
