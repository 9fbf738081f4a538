"""Host pieces of bench.py's JSON line: every roofline entry carries the keys the line promises
(bound, achieved, peak, unit, frac, traffic) with achieved / peak = frac; the ALU view of the
hypothesis search counts tries against the derived issue peak; the HBM views count algorithmic
bytes per pixel; the peaks fall back to the stated figures without the measured-peaks file."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = {"bound", "achieved", "peak", "unit", "frac", "traffic"}


@pytest.mark.parametrize("stage", ["query_raycast", "forest_eval", "forest_hypotheses", "forest_verify"])
def test_roofline_entries_carry_the_promised_keys(stage):
    r = bench.roofline(stage, 12.5, 256, 1.3e9, {"sm_max_mhz": 2070.0}, 152)
    assert KEYS <= set(r) and r["bound"] in ("hbm", "alu") and r["limiter"]
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    json.dumps(r)                                        # serialisable as it stands


def test_alu_view_counts_tries_against_the_derived_peak():
    r = bench.roofline("forest_hypotheses", 20.0, 256, 2.0e9, {"sm_max_mhz": 2000.0}, 148)
    assert r["unit"] == "Gtries/s" and r["achieved"] == pytest.approx(2.0e9 / 0.02 / 1e9)
    assert r["peak"] == pytest.approx(bench.IMAD_PER_CLK_SM * 148 * 2000e6 / bench.IMAD_PER_TRY / 1e9)


def test_hbm_view_counts_algorithmic_bytes_per_pixel():
    r = bench.roofline("query_raycast", 10.0, 100, 0, None, 152)
    want = bench.ALG_BYTES_PER_PIXEL["query_raycast"] * bench.W * bench.H * 100 / 0.01 / 1e9
    assert r["unit"] == "GB/s" and r["achieved"] == pytest.approx(want)
    per = bench.PROFILED_TRAFFIC_BYTES_PER_ATTEMPT["query_raycast"]
    assert r["traffic"] == (None if per is None else pytest.approx(per * 100))


def test_peaks_fall_back_without_the_measured_file(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    assert bench.bf16_peaks() == (1900.0, 1700.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": 2000.0,
                                                              "bf16_tflops_sustained": 1800.0}))
    assert bench.measured_peaks() == (7000.0, "measured")
    assert bench.bf16_peaks() == (2000.0, 1800.0, "measured")
