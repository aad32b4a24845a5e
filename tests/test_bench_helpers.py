"""Host-side pieces of the benchmark's JSON line that need no GPU: the batched FP32 leg's HBM
roofline (algorithmic 40 B per member-update against the measured copy bandwidth, or the
fallback figure when no measured peak is at hand)."""
import json

import bench


def test_batched_roofline_uses_the_measured_peak(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.batched_roofline(7.5e10)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == 3000.0  # 40 B x 7.5e10 / s
    assert r["peak"] == 6000.0 and r["frac"] == 0.5
    assert r["peak_source"].startswith("of measured")


def test_batched_roofline_falls_back_without_a_peak_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.batched_roofline(1.7e11)
    assert r["peak"] == bench.HBM_FALLBACK_GBS and r["peak_source"].startswith("of fallback")
    assert abs(r["frac"] - 40.0 * 1.7e11 / 1e9 / bench.HBM_FALLBACK_GBS) < 1e-12
