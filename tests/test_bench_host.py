"""Host-side arithmetic of the benchmark line: the roofline of the dominant
kernel (bound, achieved over peak, the measured DRAM traffic where a capture
exists) and the workload config shared by both arms."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6651.0, "sm_max_mhz": 2070.0}
T63 = "t63_192x96x29_n80_r2"


def test_alu_bound_dominant_kernel():
    prof = {"regress": (2, 13.0), "bandchol": (1, 3.8), "anomalies": (1, 0.1)}
    work = {"regress": (11.3e9, 256.6e6), "bandchol": (1.0e9, 2.14e9), "anomalies": (1e6, 3e8)}
    r = bench.roofline(prof, work, PEAKS, "measured", 2070.0, True, T63, "fp32")
    assert r["kernel"] == "regress" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["avg_launch_ms"] == pytest.approx(6.5)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(11.3e9 / 6.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == bench.TRAFFIC_PER_LAUNCH[("regress", T63, "fp32")]
    assert r["algorithmic_per_launch"] == {"flops": 11.3e9, "bytes": 256.6e6}


def test_hbm_bound_kernel_and_no_capture():
    prof = {"writeback": (3, 0.9)}
    work = {"writeback": (1e6, 1.0e9)}
    r = bench.roofline(prof, work, PEAKS, "measured", None, True, T63, "fp32")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6651.0
    assert r["achieved"] == pytest.approx(1.0e9 / 0.3e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6651.0)
    assert r["traffic"] is None  # no capture of this kernel


def test_fp64_peak_and_other_workload_has_no_traffic():
    prof = {"regress": (1, 50.0)}
    work = {"regress": (5e9, 1e8)}
    r = bench.roofline(prof, work, PEAKS, "measured", 2070.0, False, T63, "fp64")
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_NOMINAL_TFLOPS
    assert r["traffic"] is None


def test_both_arms_share_the_config():
    sys.argv = ["bench.py", "--impl", "reference"]
    args = bench.parse_args()
    from synthetic import WORKLOADS
    w = WORKLOADS[args.workload]
    c1, c2 = bench.workload_config(args, w, 1), bench.workload_config(args, w, 2)
    assert c1["workload"] == args.workload and c1["n"] == w.n and c1["N"] == w.N
    assert c1["parallelism"] == "1 GPU" and c2["parallelism"] == "independent problem per GPU"
