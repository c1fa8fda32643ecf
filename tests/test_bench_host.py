"""Host-side arithmetic of the benchmark line: the roofline of the dominant
kernel (bound, achieved over peak, the measured DRAM traffic where a capture
exists) and the workload config shared by both arms."""
import os
import sys

import numpy as np
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
    r = bench.roofline(prof, work, PEAKS, "measured", 2070.0, True, T63, "fp32", 152)
    assert r["kernel"] == "regress" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["avg_launch_ms"] == pytest.approx(6.5)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(11.3e9 / 6.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == bench.TRAFFIC_PER_LAUNCH.get(("regress", T63, "fp32"))
    assert r["algorithmic_per_launch"] == {"flops": 11.3e9, "bytes": 256.6e6}


def test_hbm_bound_kernel_and_no_capture():
    prof = {"writeback": (3, 0.9)}
    work = {"writeback": (1e6, 1.0e9)}
    r = bench.roofline(prof, work, PEAKS, "measured", None, True, T63, "fp32", 152)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6651.0
    assert r["achieved"] == pytest.approx(1.0e9 / 0.3e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6651.0)
    assert r["traffic"] is None  # no capture of this kernel


def test_fp64_peak_and_other_workload_has_no_traffic():
    prof = {"regress": (1, 50.0)}
    work = {"regress": (5e9, 1e8)}
    r = bench.roofline(prof, work, PEAKS, "measured", 2070.0, False, T63, "fp64", 152)
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


def test_sm_count_enters_the_alu_peak():
    prof = {"regress": (1, 5.0)}
    work = {"regress": (1e10, 1e6)}
    a = bench.roofline(prof, work, PEAKS, "measured", 2000.0, True, T63, "fp32", 152)
    b = bench.roofline(prof, work, PEAKS, "measured", 2000.0, True, T63, "fp32", 160)
    assert b["peak"] == pytest.approx(a["peak"] * 160 / 152)
    assert b["frac"] == pytest.approx(a["frac"] * 152 / 160)


def test_path_roofline_sums_per_kernel_bounds():
    """Path fraction = sum of per-kind roofline times / sum of measured times; the
    tensor-core kinds take the TF32 rate over three, the others the FP32 lanes."""
    peaks = {"hbm_gbs": 5000.0, "bf16_tflops": 1800.0}
    steps = 2
    prof = {"regress": (2, 10.0), "bandchol": (2, 8.0), "writeback": (2, 1.0), "rhs": (0, 0.0)}
    work = {"regress": (8.0e9, 1e6), "bandchol": (3.0e11, 2.0e9), "writeback": (0.0, 1.0e9),
            "rhs": (1.0, 1.0)}
    r = bench.path_roofline(prof, work, peaks, 2000.0, True, 100, steps, {"bandchol"})
    alu = 100 * 128 * 2 * 2000e6 / 1e12
    tpk = 1800.0 / 2 / 3
    want = {"regress": 2 * 8.0e9 / (alu * 1e12) * 1e3 / steps,
            "bandchol": 2 * max(3.0e11 / (tpk * 1e12), 2.0e9 / 5e12) * 1e3 / steps,
            "writeback": 2 * 1.0e9 / 5e12 * 1e3 / steps}
    for k, v in want.items():
        assert r["per_kernel"][k]["roofline_ms"] == pytest.approx(v)
    assert "rhs" not in r["per_kernel"]
    assert r["measured_ms_per_step"] == pytest.approx(19.0 / steps)
    assert r["path_frac"] == pytest.approx(sum(want.values()) / (19.0 / steps))


def _slot_offsets(r, vr, periodic):
    """Stencil slot order of the library (lower levels' boxes, the r earlier rows,
    the r left neighbours, then the r seam neighbours), restated for this test."""
    w = 2 * r + 1
    out = [(-vr + s // (w * w), (s % (w * w)) // w - r, s % w - r) for s in range(vr * w * w)]
    out += [(0, -r + s // w, s % w - r) for s in range(r * w)]
    out += [(0, 0, -r + s) for s in range(r)]
    if periodic:
        out += [(0, 0, 1 + s) for s in range(r)]
    return tuple(np.array(c, dtype=np.int32) for c in zip(*out))


def test_cpu_sample_leg_and_accuracy_report(tmp_path):
    """The CPU-baseline child times the oracle on a sample and stores its values;
    the accuracy report of outputs equal to the oracle's is zero, and a planted
    error in one D entry and one analysis value shows up in D and X^a."""
    import oracle as O
    from synthetic import WORKLOADS, make_inputs
    w = WORKLOADS["tiny_32x16_n20_r2"]
    ref = str(tmp_path / "ref.npz")
    d = bench.run_cpu_sample(w.name, "fp64", 60, 1, 2, out=ref, steps=2)
    assert "error" not in d, d
    assert len(d["cycles_s"]) == 2 and d["workers"] == 2 and d["cycle_s"] > 0
    inp = make_inputs(w)
    g = O.Grid.from_workload(w)
    U = O.anomalies(inp.Xb.T)
    dk, dy, dx = _slot_offsets(w.r, 0, True)

    class H:
        def slot_offsets(self):
            return dk, dy, dx
    T = np.zeros((w.n, len(dk)))
    D = np.zeros(w.n)
    for j, P, beta, dj in O.estimate_rows(g, U, range(w.n), w.ridge_c):
        v, k, y, x = g.coords(j)
        coef = {q: -b for q, b in zip(P, beta)}
        for s in range(len(dk)):
            yy, xx = y + dy[s], (x + dx[s]) % w.nlon
            if 0 <= yy < w.nlat and k + dk[s] >= 0:
                T[j, s] = coef.get(g.label(v, k + dk[s], yy, xx), 0.0)
        D[j] = dj
    Xa = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    acc = bench.accuracy_report(w, ref, inp.Xb, T, D, Xa, H())
    assert max(acc[k] for k in ("T", "D", "D_elementwise", "dX", "Xa")) < 1e-12, acc
    z = np.load(ref)
    D2, Xa2 = D.copy(), Xa.copy()
    D2[int(z["rows"][3])] *= 1.001
    i0 = int(z["sd"][0])
    Xa2[0, int(z[f"int{i0}"][0])] += 0.5
    acc = bench.accuracy_report(w, ref, inp.Xb, T, D2, Xa2, H())
    assert acc["D_elementwise"] == pytest.approx(1e-3, rel=1e-6)
    assert acc["Xa"] > 1e-3 and acc["T"] < 1e-12
