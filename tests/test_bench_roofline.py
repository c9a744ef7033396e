"""The benchmark's roofline arithmetic on the CPU: the derived ALU peaks, the
bound each kernel class is measured against, and the rule that an ncu
traffic figure is reported only for the kernel source it was taken on."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = dict(hbm=6689.5, bf16=1929.0, src="measured", sm_mhz=2070.0, sms=152)


def test_alu_peaks_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz; FP64 at the part's rate
    assert bench.alu_peak_tflops("f32", 2070.0, 152) == pytest.approx(80.54784)
    assert bench.alu_peak_tflops("f32", 1035.0, 76) == pytest.approx(80.54784 / 4)
    assert bench.alu_peak_tflops("fp64", 2070.0, 152) == 1.25


def test_each_class_against_its_bound():
    d = dict(ms=2.0, bytes=6.0e9, flops=4.0e10)
    hbm = bench.class_roofline("schur", d, PEAKS, "f32")
    assert hbm["bound"] == "hbm" and hbm["achieved"] == pytest.approx(3000.0)
    assert hbm["frac"] == pytest.approx(3000.0 / 6689.5)
    alu = bench.class_roofline("id", d, PEAKS, "f32")
    assert alu["bound"] == "alu" and alu["achieved"] == pytest.approx(20.0)
    assert alu["peak"] == pytest.approx(80.54784)
    # the residual operator is FP64 whatever the factor's precision; the
    # products inside GMRES follow the factor's
    assert bench.class_roofline("refine_op", d, PEAKS, "f32")["peak"] == 1.25
    assert bench.class_roofline("inner_op", d, PEAKS, "f32")["peak"] == pytest.approx(80.54784)
    assert bench.class_roofline("id", dict(ms=0.0, bytes=0.0, flops=0.0), PEAKS, "f32") is None


def test_traffic_only_for_the_source_it_was_taken_on(monkeypatch):
    with open(os.path.join(ROOT, "paper_1609_08130_gb300", "csrc", "kernels.cu"), "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    table = {"now": {"bytes_per_launch": 1.0e6, "kernels_sha256": sha},
             "stale": {"bytes_per_launch": 2.0e6, "kernels_sha256": "0" * 64}}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", table)
    assert bench.ncu_traffic("now") == 1.0e6
    assert bench.ncu_traffic("stale") is None
    assert bench.ncu_traffic("absent") is None
