"""Host-side logic of bench.py (no GPU): the traffic record is tied to the pass kernel's
source, the roofline peaks come from the measured file, and the clock sampler's summary
reads nvidia-smi's CSV lines (median SM clock, throttle reasons seen)."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_the_committed_pass_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "aca_cols_pass_traffic.json")))
    src = open(os.path.join(ROOT, "paper_2502_11017_gb300", "csrc", "aca.cu"), "rb").read()
    assert rec["source_sha256"] == hashlib.sha256(src).hexdigest(), \
        "aca.cu changed since its DRAM traffic was captured: recapture it"
    t = bench.traffic_record()
    assert t == rec["traffic_bytes_per_launch"]
    # read + write of the captured case, scaled by the rows of the bench matrix
    assert t == (rec["captured_dram_bytes_read"] + rec["captured_dram_bytes_write"]) * rec["scale_to_65536x8192"]
    # within 2 % of the algorithmic bytes (one read of A per launch)
    assert abs(t / rec["algorithmic_bytes_per_launch"] - 1.0) < 0.02


def test_traffic_record_is_dropped_when_the_source_differs(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    csrc = tmp_path / "paper_2502_11017_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "aca.cu").write_text("// another source\n")
    rec = json.load(open(os.path.join(ROOT, "profiles", "aca_cols_pass_traffic.json")))
    (prof / "aca_cols_pass_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record() is None


def test_peaks_come_from_the_measured_file():
    peaks, kind = bench.measured_peaks()
    assert kind == "measured"
    assert peaks["hbm_gbs"] > 1000.0 and peaks["bf16_tflops"] > 100.0


def test_clock_summary_median_and_reasons():
    s = bench.ClockSampler(0)
    s.out = "\n".join([
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
