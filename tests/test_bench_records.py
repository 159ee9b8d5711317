"""bench.py's use of the committed ncu records: a record counts only while
the kernel sources hash to its sources_sha256, and the batched form's issue
roofline is the record's warp instructions against 4 per SM cycle."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def write_record(path, sha, inst=4000, scale=2):
    with open(path, "w") as f:
        f.write("# test record\n")
        f.write(f"sources_sha256: {sha}\n")
        f.write(f"scale: {scale}\n")
        f.write("stream_warp_inst: 1000\nstiff_warp_inst: 900\nfb_warp_inst: 100\n")
        f.write("stream_us: 1.0\nstiff_us: 2.0\nfb_us: 0.5\n")
        f.write(f"warp_inst_per_step: {inst}\n")
        f.write("shape: 1,8,0\n")


def test_issue_roofline_from_a_current_record(tmp_path, monkeypatch):
    p = tmp_path / "issue.txt"
    write_record(p, bench.kernel_sources_hash())
    monkeypatch.setattr(bench, "ISSUE_FILE", str(p))
    r = bench.batched_issue_roofline(ms=1e-3, sm_mhz=1000.0, num_sms=2)
    # 4000 warp instructions in 1 us against 2 SMs x 4 x 1 GHz = 8e9 / s
    assert r["bound"] == "issue"
    assert r["achieved"] == pytest.approx(4.0)  # G warp instructions / s
    assert r["peak"] == pytest.approx(8.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["launch_shape"] == [1, 8, 0] and bench.recorded_issue_shape() == (1, 8, 0)
    k = r["kernels"]["ion_stiff_kernel"]
    assert k["warp_inst_per_step"] == pytest.approx(1800)
    assert k["issue_frac_in_capture"] == pytest.approx(900 / 2e-6 / 8e9)


def test_stale_records_are_not_used(tmp_path, monkeypatch):
    p = tmp_path / "issue.txt"
    write_record(p, "0" * 64)
    monkeypatch.setattr(bench, "ISSUE_FILE", str(p))
    assert bench.batched_issue_roofline(ms=1.0, sm_mhz=2000.0, num_sms=152) is None
    assert bench.recorded_issue_shape() is None
    t = tmp_path / "traffic.txt"
    t.write_text("sources_sha256: " + "0" * 64 + "\ndram_bytes_per_step: 123\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(t))
    assert bench.recorded_traffic() is None
    t.write_text(f"sources_sha256: {bench.kernel_sources_hash()}\ndram_bytes_per_step: 123\n")
    assert bench.recorded_traffic() == 123


def test_no_roofline_without_a_clock(tmp_path, monkeypatch):
    p = tmp_path / "issue.txt"
    write_record(p, bench.kernel_sources_hash())
    monkeypatch.setattr(bench, "ISSUE_FILE", str(p))
    assert bench.batched_issue_roofline(ms=1.0, sm_mhz=None, num_sms=152) is None
