"""Host-side arithmetic of bench.py (no GPU): the roofline of the dominant kernel class, the
per-class breakdown, the ncu traffic lookup keyed by the kernel source, and the timing defaults."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


def cls(launches, ms, bytes_, flops=0.0, bytes_pass=None):
    return {"launches": launches, "ms": ms, "bytes": bytes_, "flops": flops,
            "bytes_pass": bytes_ if bytes_pass is None else bytes_pass}


def test_roofline_takes_the_dominant_class_and_divides_bytes_per_launch_by_its_mean_time():
    prof = {"update_norm": cls(10, 1.0, 10 * 500e6), "mdot": cls(10, 0.8, 10 * 480e6), "small": cls(40, 0.2, 0.0)}
    roof = bench.roofline_from_profile(prof, {"hbm_gbs": 6000.0}, "measured", 2070.0, "no-such-workload")
    assert roof["kernel_class"] == "update_norm"
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    # 500 MB per launch in 0.1 ms = 5000 GB/s
    assert roof["achieved"] == pytest.approx(5000.0)
    assert roof["frac"] == pytest.approx(5000.0 / 6000.0)
    assert roof["avg_launch_us"] == pytest.approx(100.0)
    assert roof["share_of_eager_solve"] == pytest.approx(1.0 / 2.0)
    assert roof["traffic"] is None and "no ncu capture" in roof["traffic_note"]
    assert "of measured" in roof["peak_source"]


def test_roofline_calls_an_fp64_heavy_class_alu_bound():
    # 1e9 flops over 1e8 bytes per launch is far above the FP64 ridge point (about 0.19 flop/B)
    prof = {"apply": cls(4, 4.0, 4 * 1e8, flops=4 * 1e9)}
    roof = bench.roofline_from_profile(prof, {"hbm_gbs": 6000.0}, "fallback", 2070.0)
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    peak = 2 * bench.FP64_FMA_PER_SM_CLK * bench.SM_COUNT * 2070.0 * 1e6 / 1e12
    assert roof["peak"] == pytest.approx(peak)
    assert roof["achieved"] == pytest.approx(1e9 / 1e-3 / 1e12)  # 1 GFLOP per 1 ms launch
    assert roof["hbm_gbs_achieved"] == pytest.approx(1e8 / 1e-3 / 1e9)


def test_breakdown_reports_pass_by_pass_bytes_only_for_blocked_kernels():
    prof = {"smooth_fine": cls(2, 0.02, 2 * 27e6, bytes_pass=2 * 73e6), "apply": cls(2, 0.03, 2 * 33e6),
            "unused": cls(0, 0.0, 0.0)}
    out = bench.breakdown_from_profile(prof, 6000.0)
    assert "unused" not in out
    assert out["apply"]["GB/s"] == pytest.approx(2 * 33e6 / 0.03e-3 / 1e9, rel=1e-3)
    assert "GB/s_per_pass" not in out["apply"]
    assert out["smooth_fine"]["GB/s_per_pass"] == pytest.approx(2 * 73e6 / 0.02e-3 / 1e9, rel=1e-3)
    assert out["smooth_fine"]["frac_per_pass"] == pytest.approx(out["smooth_fine"]["GB/s_per_pass"] / 6000.0, rel=1e-3)


def test_ncu_traffic_is_reported_only_while_the_captured_source_is_unchanged(monkeypatch):
    src = "paper_1012_4307_gb300/csrc/kernels_gs_df.cu"
    with open(os.path.join(ROOT, src), "rb") as fh:
        sha = hashlib.sha1(fh.read()).hexdigest()
    entry = dict(kernel="k", source=src, sha1=sha, bytes=123, launch="slot 1", profile="profiles/x.md")
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w", "c"), entry)
    assert bench.ncu_traffic("w", "c")[0] == 123
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w", "c"), dict(entry, sha1="0" * 40))
    traffic, note = bench.ncu_traffic("w", "c")
    assert traffic is None and "changed" in note


def test_every_traffic_entry_names_an_existing_source_and_profile():
    for (workload, kclass), t in bench.NCU_TRAFFIC.items():
        assert workload in bench.WORKLOADS
        assert os.path.exists(os.path.join(ROOT, t["source"]))
        assert os.path.exists(os.path.join(ROOT, t["profile"]))
        assert t["bytes"] > 0 and len(t["sha1"]) == 40


def test_timing_defaults_keep_at_least_three_warmup_steps():
    args = bench.parse([])
    assert args.warmup >= 3 and args.steps >= 1 and args.gpus == 1
    assert args.workload == bench.WORKLOADS[0]
