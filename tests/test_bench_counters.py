"""bench.py's use of the committed ncu counters (CPU): they are reported only
while the projector source they were taken on is unchanged, and the
instruction-issue roofline is their warp instructions over the live time
against 4 warp instructions per clock on each of the 152 SMs."""
import json

import pytest

import bench


def test_counters_follow_the_projector_source(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "paper_2110_13526_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "projector.cu").write_bytes(b"kernel source v1\n")
    import hashlib
    sha = hashlib.sha256(b"kernel source v1\n").hexdigest()
    ent = {"dram_bytes_per_launch": 1.0e9, "projector_sha256": sha, "issue_active": 0.5,
           "warp_inst_per_launch": 2.0e9, "red_sectors_per_launch": 4.0e8}
    (root / "profiles" / "traffic.json").write_text(json.dumps({"k_backward_cm": ent}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_counters("k_backward_cm") == ent
    assert bench.traffic_for("k_backward_cm") == 1.0e9
    assert bench.ncu_counters("k_forward_cm") is None
    # a changed source invalidates every committed counter
    (src / "projector.cu").write_bytes(b"kernel source v2\n")
    assert bench.ncu_counters("k_backward_cm") is None
    assert bench.traffic_for("k_backward_cm") is None
    assert bench.issue_roofline(bench.ncu_counters("k_backward_cm") or {}, 0.01, None) is None


def test_issue_roofline_arithmetic():
    ent = {"warp_inst_per_launch": 1.0e10, "red_sectors_per_launch": 3.0e9}
    r = bench.issue_roofline(ent, 0.010, {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0})
    peak = 4 * 152 * 2000e6
    assert r["bound"] == "alu" and r["unit"] == "warp-inst/s"
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(1.0e12)
    assert r["frac"] == pytest.approx(1.0e12 / peak)
    assert r["l2_reduction_sectors_per_s"] == pytest.approx(3.0e11)
    # no clock sample: the maximum clock, else 2070 MHz
    assert bench.issue_roofline(ent, 0.010, {"sm_mhz": None, "sm_max_mhz": 1980.0})["peak"] == \
        pytest.approx(4 * 152 * 1980e6)
    assert bench.issue_roofline(ent, 0.010, None)["peak"] == pytest.approx(4 * 152 * 2070e6)
    assert "l2_reduction_sectors_per_s" not in bench.issue_roofline(
        {"warp_inst_per_launch": 1.0e10}, 0.010, None)
