#!/usr/bin/env python3
"""Throughput of the EnKF-MC analysis step on GB300: analysis cycles per second.

One step = one analysis cycle of the whole hot path on one synthetic ensemble
already resident in HBM: enkfmc_estimate (anomalies + the regressions of every
component), enkfmc_assemble (boundary re-estimation, band assembly, banded
Cholesky of every sub-domain block) and enkfmc_analyze (right-hand sides,
N-member band solves with refinement, interior write-back).  Workload: the
T63-shaped state (192 x 96 x (7 levels x 4 variables + 1), n = 534,528),
N = 80 members, r = 2, 12 x 12 sub-domains with an r-wide boundary, 50% of the
components observed; FP32 by default.  Inputs are larger than L2 (X^b alone is
171 MB in FP32), so no flush is needed between steps.

The headline steps run with the library's per-kernel events off; a second
timed pass with them on gives the per-kernel split, the roofline of the
dominant kernel and the path fraction (sum of per-kernel roofline times over
the cycle time).  Also printed: the end-to-end rate through enkfmc_cycle_host
from pinned host buffers, the SM clocks seen during the timed region, and the
CPU baseline: the FP64 oracle timed on a bounded sample on one host thread and
on all host cores; the oracle values of that sample give the accuracy report
(max relative error of T, D, dX and X^a against the oracle).  Side lines: the
plain FP64 form, forward + adjoint (T63 with N = 80 and with N = 40), the batch
of uneven problems, filter cycling, the accuracy study, and the dual form
against the primal form on sparse networks (4% and 10% of the components
observed).
Multi-GPU (torchrun): every rank runs an independent problem (its own seed);
value = cycles of all ranks / slowest rank's time.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EnKF-MC analysis cycles/sec at T63 shape (N=80); % roofline; fwd+adj vs plain"
WORKLOAD = "t63_192x96x29_n80_r2"
ADJ_WORKLOAD = "t63_192x96x29_n40_r2"
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture of its current version on the named workload and
# precision (the capture commands are in profiles/); a kernel without one
# reports null.
TRAFFIC_PER_LAUNCH = {
    # the global-rows launch of the tiled single-precision kernel
    ("regress", "t63_192x96x29_n80_r2", "fp32"): 724_083_968,
}
TUNING_CACHE = os.path.join(ROOT, "paper_1606_00807_gb300", "tuning_gb300.json")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-FP64 and forward+adjoint side measurements")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="host processes of the all-cores oracle leg (0: every core)")
    ap.add_argument("--sample-rows", type=int, default=250)
    ap.add_argument("--sample-subdomains", type=int, default=1)
    ap.add_argument("--sample-out", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--sample-steps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--t127-only", action="store_true",
                    help="only the T127-shaped scale line (mixed against plain FP32)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batch of 256 uneven problems (one CUDA graph per cycle)")
    ap.add_argument("--dual-only", action="store_true",
                    help="only the dual form against the primal form (sparse networks)")
    ap.add_argument("--fwd-adj-only", action="store_true",
                    help="only forward + adjoint on the headline workload, FP32")
    ap.add_argument("--tune", action="store_true",
                    help="autotune every batch shape missing from the tuning cache")
    ap.add_argument("--tune-max", type=int, default=64,
                    help="with --tune: the most expensive shapes tuned (the rest keep defaults)")
    ap.add_argument("--tuning", default=TUNING_CACHE,
                    help="tuning cache (JSON) read, and with --tune written")
    return ap.parse_args(argv)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (bounded sample): the cpu_baseline leg and --impl reference.
# The sample's oracle values also serve as the reference of the accuracy report.
# ----------------------------------------------------------------------------
def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def sample_plan(n, nsd, nrows, nsub, seed=0):
    """The sampled rows (of n) and sub-domains (of nsd) of one step (deterministic)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, min(nrows, n), replace=False))
    picks = [int(i) for i in rng.choice(nsd, min(nsub, nsd), replace=False)]
    return rows, picks


_CTX = {}


def _oracle_rows(rows):
    import oracle as O
    c = _CTX
    t0 = time.perf_counter()
    out = O.estimate_rows(c["g"], c["U"], rows, c["w"].ridge_c)
    return time.perf_counter() - t0, [(j, list(P), beta, d) for j, P, beta, d in out]


def _oracle_subdomain(i):
    import oracle as O
    c = _CTX
    sd = c["sds"][i]
    t0 = time.perf_counter()
    dX = O.local_analysis(c["g"], sd, c["U"], c["Xb"], c["Ys"], c["inp"].R, c["inp"].obs_idx,
                          c["w"].ridge_c)
    dt = time.perf_counter() - t0
    pos = {int(q): k for k, q in enumerate(sd.ext)}
    rows = [pos[int(q)] for q in sd.interior]
    return dt, i, c["Xb"][sd.interior] + dX[rows]


def cpu_sample_main(args):
    """Child process: time the FP64 oracle on bounded samples (--sample-steps of
    them, each on its own rows and sub-domains) and print one JSON line; with
    --sample-out also store the first sample's oracle values (and the interiors
    of its sub-domains).  This process never initialises CUDA, so its worker
    pool may fork."""
    import multiprocessing as mp

    import numpy as np
    import oracle as O
    from synthetic import WORKLOADS, make_inputs
    w = WORKLOADS[args.workload]
    dt = np.float64 if args.precision == "fp64" else np.float32
    inp = make_inputs(w, dt)
    workers = max(1, args.cpu_workers)
    Xb = inp.Xb.T.astype(np.float64)
    t0 = time.perf_counter()
    U = O.anomalies(Xb)
    t_anom = time.perf_counter() - t0
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    _CTX.update(g=g, sds=sds, U=U, Xb=Xb, Ys=Ys, inp=inp, w=w)
    pool = mp.get_context("fork").Pool(workers) if workers > 1 else None
    if pool:
        pool.map(abs, range(4 * workers))              # every worker up before timing
    run = pool.map if pool else lambda f, xs: [f(x) for x in xs]
    cycles = []
    for step in range(max(1, args.sample_steps)):
        rows, picks = sample_plan(g.n, len(sds), args.sample_rows * workers,
                                  args.sample_subdomains * workers, seed=step)
        chunks = [rows[k::workers] for k in range(workers)]
        t0 = time.perf_counter()
        row_res = run(_oracle_rows, chunks)
        t_rows = time.perf_counter() - t0
        t0 = time.perf_counter()
        sd_res = run(_oracle_subdomain, picks)
        t_sd = time.perf_counter() - t0
        cycles.append(t_anom + t_rows * g.n / len(rows) + t_sd * len(sds) / len(picks))
        if step == 0 and args.sample_out:
            ref = sorted((r for _, part in row_res for r in part), key=lambda r: r[0])
            width = max([len(r[1]) for r in ref] + [1])
            np.savez(args.sample_out,
                     rows=np.array([r[0] for r in ref], dtype=np.int64),
                     P=np.array([r[1] + [-1] * (width - len(r[1])) for r in ref], dtype=np.int64),
                     beta=np.array([list(r[2]) + [0.0] * (width - len(r[2])) for r in ref]),
                     D=np.array([r[3] for r in ref]),
                     sd=np.array([i for _, i, _ in sd_res], dtype=np.int64),
                     **{f"Xa{i}": x for _, i, x in sd_res},
                     **{f"int{i}": sds[i].interior for _, i, _ in sd_res})
    if pool:
        pool.close()
        pool.join()
    print(json.dumps({"cycle_s": cycles[0], "cycles_s": cycles, "workers": workers,
                      "sample": f"{len(rows)} of {g.n} regressions + {len(picks)} of {len(sds)} "
                                f"sub-domain analyses"}))


def run_cpu_sample(workload, precision, rows, subdomains, workers, out=None, steps=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload,
           "--precision", precision, "--sample-rows", str(rows),
           "--sample-subdomains", str(subdomains), "--cpu-workers", str(workers),
           "--sample-steps", str(steps)]
    if out:
        cmd += ["--sample-out", out]
    p = subprocess.run(cmd, capture_output=True, text=True, env=env)
    if p.returncode != 0:
        tail = p.stderr.strip().splitlines()
        return {"error": tail[-1] if tail else "failed"}
    return json.loads(p.stdout.strip().splitlines()[-1])


def cpu_baseline(args, out=None, workload=None):
    """The FP64 oracle on the host cores: one thread and every core (one process
    per core, each on its share of the sampled rows and one sub-domain), cycle
    time extrapolated to the full workload.  `out`: where the all-cores leg
    stores its oracle values (the accuracy reference)."""
    workload = workload or args.workload
    ncores = args.cpu_workers or os.cpu_count() or 1
    one = run_cpu_sample(workload, args.precision, 4 * args.sample_rows,
                         args.sample_subdomains, 1)
    allc = run_cpu_sample(workload, args.precision, args.sample_rows, args.sample_subdomains,
                          ncores, out)
    res = {"unit": "cycles/s", "kind": "oracle", "cpu_model": cpu_model(),
           "nproc": os.cpu_count()}
    if "error" in allc or "error" in one:
        res["error"] = allc.get("error") or one.get("error")
        return res
    res.update({"value": 1.0 / allc["cycle_s"], "cores": allc["workers"],
                "sample": allc["sample"] + " per step, one process per core (FP64 numpy/scipy "
                          "oracle, one thread each); cycle time extrapolated to the workload",
                "single_thread": {"value": 1.0 / one["cycle_s"], "cores": 1,
                                  "sample": one["sample"]}})
    return res


def accuracy_report(w, ref_path, Xb, T, D, Xa, handle):
    """Max relative errors of the GPU outputs against the oracle values the CPU
    baseline leg stored: T (off-diagonal, per variable), D (per variable and element
    by element), and dX, X^a on the sampled sub-domains' interiors (per variable;
    max |x - x_ref| / max |x_ref|)."""
    import numpy as np
    from synthetic import variable_of
    d = np.load(ref_path)
    rows = d["rows"]
    dk, dy, dx = handle.slot_offsets()
    # label of each stencil slot of each sampled row (ring longitude)
    nvl = [w.var_levels(v) for v in range(w.nvar)]
    var = variable_of(w, rows)
    off = np.array([w.var_offset(v) for v in range(w.nvar)])
    rem = rows - off[var]
    k, rem = rem // (w.nlat * w.nlon), rem % (w.nlat * w.nlon)
    y, x = rem // w.nlon, rem % w.nlon
    kk, yy, xx = k[:, None] + dk[None], y[:, None] + dy[None], x[:, None] + dx[None]
    ok = (kk >= 0) & (kk < np.array(nvl)[var][:, None]) & (yy >= 0) & (yy < w.nlat)
    if w.lon_periodic:
        xx = xx % w.nlon
    else:
        ok &= (xx >= 0) & (xx < w.nlon)
    lab = off[var][:, None] + (kk * w.nlat + yy) * w.nlon + xx
    Tg = T[rows].astype(np.float64)
    Tr = np.zeros_like(Tg)
    for a in range(len(rows)):
        coef = {int(q): -b for q, b in zip(d["P"][a], d["beta"][a]) if q >= 0}
        for s in range(len(dk)):
            if ok[a, s]:
                Tr[a, s] = coef.get(int(lab[a, s]), 0.0)

    def per_var(got, ref, v):
        worst = 0.0
        for u in np.unique(v):
            sel = v == u
            den = np.abs(ref[sel]).max()
            if den > 0:
                worst = max(worst, float(np.abs(got[sel] - ref[sel]).max() / den))
        return worst

    Dg = D[rows].astype(np.float64)
    out = {"T": per_var(Tg, Tr, var), "D": per_var(Dg, d["D"], var),
           "D_elementwise": float(np.max(np.abs(Dg - d["D"]) / np.abs(d["D"])))}
    eX = edX = 0.0
    for i in d["sd"]:
        lab_i = d[f"int{int(i)}"]
        v = variable_of(w, lab_i)
        ref = d[f"Xa{int(i)}"]
        got = Xa[:, lab_i].T.astype(np.float64)
        xb = Xb[:, lab_i].T.astype(np.float64)
        eX = max(eX, per_var(got, ref, v))
        edX = max(edX, per_var(got - xb, ref - xb, v))
    out.update({"dX": edX, "Xa": eX,
                "sample": f"{len(rows)} rows, sub-domains {[int(i) for i in d['sd']]}"})
    return out


# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def alu_peak(fp32, sm_count, sm_max_mhz):
    """(TFLOP/s, note) of the arithmetic pipe: FP32 FMA lanes at the maximum SM
    clock, or the FP64 nominal rate."""
    if fp32:
        return (sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12,
                f"FP32 FMA: {sm_count} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                f"{sm_max_mhz:.0f} MHz")
    return FP64_NOMINAL_TFLOPS, "FP64 nominal 1.25 TFLOP/s"


def roofline(prof, work, peaks, peak_src, sm_max_mhz, fp32, workload, precision, sm_count):
    """Roofline of the dominant kernel (largest device time per cycle).

    prof: kind -> (calls, ms); work: kind -> (flops, bytes) per call.  The bound
    is the one whose time per call is larger at its peak: the arithmetic pipe
    (alu_peak) for flops, the measured copy bandwidth for bytes; achieved = the
    algorithmic work per call over the kind's average call time."""
    dom = max(prof, key=lambda k: prof[k][1])
    launches, dom_ms = prof[dom]
    avg_s = dom_ms / max(1, launches) / 1e3
    flops, nbytes = work[dom]
    sm_max = sm_max_mhz or peaks.get("sm_max_mhz", 2070.0)
    apeak, anote = alu_peak(fp32, sm_count, sm_max)
    t_alu = flops / (apeak * 1e12)
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    if t_alu >= t_hbm:
        achieved = flops / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": apeak, "unit": "TFLOP/s",
                "frac": achieved / apeak, "peak_source": f"derived: {anote}"}
    else:
        achieved = nbytes / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peak_src} hbm_gbs"}
    roof["traffic"] = TRAFFIC_PER_LAUNCH.get((dom, workload, precision))
    roof["kernel"] = dom
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["algorithmic_per_launch"] = {"flops": flops, "bytes": nbytes}
    return roof


def path_roofline(prof, work, peaks, sm_max_mhz, fp32, sm_count, steps, tensor_kinds):
    """Sum over kernel kinds of the roofline time (calls x max(flops / pipe peak,
    bytes / HBM peak)) against the measured time of the same calls, per step.
    The pipe of `tensor_kinds` (band Cholesky and solves on the tensor cores) is
    the TF32 rate (half the measured bf16 rate) over 3, the products per
    FP32-accurate product of their split operands; every other kind's is
    alu_peak."""
    sm_max = sm_max_mhz or peaks.get("sm_max_mhz", 2070.0)
    apeak, _ = alu_peak(fp32, sm_count, sm_max)
    tpeak = peaks.get("bf16_tflops", 1900.0) / 2.0 / 3.0
    per, t_roof, t_meas = {}, 0.0, 0.0
    for k, (calls, ms) in prof.items():
        if not calls:
            continue
        flops, nbytes = work[k]
        pipe = tpeak if k in tensor_kinds else apeak
        rf = calls * max(flops / (pipe * 1e12), nbytes / (peaks["hbm_gbs"] * 1e9)) * 1e3 / steps
        per[k] = {"ms": ms / steps, "roofline_ms": rf,
                  "frac": rf / (ms / steps) if ms > 0 else None}
        t_roof += rf
        t_meas += ms / steps
    return {"path_frac": t_roof / t_meas if t_meas > 0 else None,
            "roofline_ms_per_step": t_roof, "measured_ms_per_step": t_meas,
            "tensor_peak_tflops": tpeak, "alu_peak_tflops": apeak, "per_kernel": per}


def workload_config(args, w, world):
    """The `config` of the JSON line (the same for both arms)."""
    esize = 8 if args.precision == "fp64" else 4
    return {"workload": args.workload, "n": w.n, "N": w.N, "r": w.r,
            "grid": f"{w.nlon}x{w.nlat}x({w.nlev}x{w.nvar_3d}+{w.nvar_2d})",
            "subdomains": f"{w.sub_lat}x{w.sub_lon}+halo{w.r}",
            "obs_frac": w.obs_frac, "precision": args.precision,
            "l2": "inputs larger than L2 (Xb %.0f MB), no flush" % (esize * w.N * w.n / 1e6),
            "parallelism": "independent problem per GPU" if world > 1 else "1 GPU"}


def rank_workload(w, rank):
    """Rank `rank`'s problem: the same shapes with its own seed (independent
    problems, no exchange between ranks)."""
    return w.with_(seed=w.seed + 17 * rank) if rank else w


def slowest_rank(x, world, device):
    """Max over ranks of a host float: the job takes as long as its slowest rank."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps, world, seconds):
    """Whole-job rate: every rank's steps over the slowest rank's time."""
    return steps * world / seconds


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synthetic import WORKLOADS
    w = WORKLOADS[args.workload]
    ncores = args.cpu_workers or os.cpu_count() or 1
    d = run_cpu_sample(args.workload, args.precision, 40, 1, ncores,
                       steps=args.warmup + args.steps)
    if "error" in d:
        print(json.dumps({"impl": "reference", "unavailable": d["error"]}))
        return
    sample = d["sample"]
    cyc = d["cycles_s"][args.warmup:]
    mean_cycle = sum(cyc) / len(cyc)
    value = 1.0 / mean_cycle
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cycles/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean_cycle * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, w, 1),
           "cpu_baseline": {"value": value, "unit": "cycles/s", "cores": ncores, "kind": "oracle",
                            "cpu_model": cpu_model(),
                            "sample": "per step: " + sample + ", one process per core; cycle "
                                      "time extrapolated"},
           "e2e": {"value": value, "unit": "cycles/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _time_steps(step, warmup, steps, stream):
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def fwd_adj_line(args, wa, ia, dev, npdt, precision, tdt, accuracy=False):
    """Forward analysis and forward + adjoint (loss 1/2 |mean(X^a) - x_ref|^2,
    dL/dX^a formed on the device, enkfmc_analyze_adjoint) on workload wa."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B

    stream = torch.cuda.Stream(device=dev)
    h = B.Handle.from_workload(wa, precision=precision, stream=stream.cuda_stream)
    h.set_observations(ia.obs_idx)
    with torch.cuda.stream(stream):
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=npdt)).to(dev, tdt)
        Xb, y, R, Z, xref = put(ia.Xb), put(ia.y), put(ia.R), put(ia.Z), put(ia.truth)
        T = torch.empty((wa.n, h.info.pmax), device=dev, dtype=tdt)
        D = torch.empty(wa.n, device=dev, dtype=tdt)
        Xa = torch.empty_like(Xb)
        Xa_bar = torch.empty_like(Xb)
        Xb_bar = torch.empty_like(Xb)
        y_bar = torch.empty_like(y)
        R_bar = torch.empty_like(R)

    def fwd():
        h.estimate(Xb, T, D)
        h.assemble(Xb, T, D, R)
        h.analyze(Xb, y, R, Z, Xa)

    def fwd_adj():
        fwd()
        with torch.cuda.stream(stream):
            Xa_bar.copy_(((Xa.mean(dim=0) - xref) / wa.N).expand_as(Xa))
        h.analyze_adjoint(Xa_bar, y_bar, R_bar, Xb_bar)

    ms_f = _time_steps(fwd, 2, 5, stream)
    ms_fa = _time_steps(fwd_adj, 1, 5, stream)
    h.profile(True)
    h.profile_read()
    _time_steps(fwd_adj, 0, 2, stream)
    prof = h.profile_read()
    h.profile(False)
    h.check("forward + adjoint steps")
    nfb = h.fp64_blocks()
    peaks, _ = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    tk = {k for k, on in (("bandchol", h.info.tc_chol), ("bandsolve", h.info.tc_solve)) if on}
    path = path_roofline(prof, h.work_per_launch(), peaks, None, precision == B.FP32, sm_count,
                         2, tk)
    line = {"workload": wa.name, "precision": "fp32" if precision == B.FP32 else "fp64",
            "fwd_cycles_per_s": 1e3 / ms_f, "fwd_adj_cycles_per_s": 1e3 / ms_fa,
            "fwd_ms": ms_f, "fwd_adj_ms": ms_fa, "adj_over_fwd": (ms_fa - ms_f) / ms_f,
            "refine_steps": h.info.refine_steps, "fp64_rows": bool(h.info.fp64_rows),
            "fp64_blocks": nfb, "blocks": h.info.nblock,
            "path_frac_fwd_adj": path["path_frac"],
            "kernels_ms_per_step": {k: v[1] / 2 for k, v in prof.items() if v[0]}}
    if accuracy and not args.no_cpu_baseline:
        fwd()
        torch.cuda.synchronize()
        ref = tempfile.mktemp(suffix=".npz")
        cb = cpu_baseline(args, out=ref, workload=wa.name)
        line["cpu_baseline"] = cb
        if os.path.exists(ref):
            line["accuracy"] = accuracy_report(wa, ref, ia.Xb, T.cpu().numpy(), D.cpu().numpy(),
                                               Xa.cpu().numpy(), h)
            os.unlink(ref)
    h.close()
    return line


def side_measurements(args, w, inp, value, dev):
    """Side lines of the headline metric, each on its own handle: the plain
    FP64 form of the same workload (cycles/s and the FP32 speed-up over it);
    forward + adjoint (the loss L = 1/2 |mean(X^a) - x_ref|^2, its gradient
    dL/dX^a formed on the device, then enkfmc_analyze_adjoint for X^b, y and
    diag(R)) against the forward analysis alone, on the same workload and at
    the T63 shape with N = 40, in FP32 (with its accuracy against the oracle)
    and in FP64 (the plain form)."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import WORKLOADS, make_inputs

    out = {}

    def guarded(key, fn):
        try:
            out[key] = fn()
        except Exception as exc:  # one side line must not hide the others
            out[key] = {"error": f"{type(exc).__name__}: {exc}"}

    guarded("plain_fp64", lambda: plain_fp64_line(w, inp, value, dev))
    guarded("fwd_adj_fp32",
            lambda: fwd_adj_line(args, w, inp, dev, np.float32, B.FP32, torch.float32))
    # forward + adjoint at the T63 shape with N = 40 (p = 37 predecessors from
    # 40 members on interior rows): FP32 with the double-precision rows, the
    # double-precision blocks and four refinement steps, against the plain FP64 form
    wa = WORKLOADS[ADJ_WORKLOAD]
    guarded("fwd_adj", lambda: fwd_adj_line(args, wa, make_inputs(wa, np.float32), dev,
                                            np.float32, B.FP32, torch.float32, accuracy=True))
    guarded("fwd_adj_plain_fp64", lambda: fwd_adj_line(args, wa, make_inputs(wa, np.float64),
                                                       dev, np.float64, B.FP64, torch.float64))
    guarded("batch", lambda: batch_line(args, dev))
    guarded("cycling", lambda: cycling_line(w, dev))
    guarded("dual", lambda: dual_line(w, dev))
    guarded("accuracy_study", lambda: accuracy_study_line(dev))
    a, b = out.get("fwd_adj", {}), out.get("fwd_adj_plain_fp64", {})
    if "fwd_adj_cycles_per_s" in a and "fwd_adj_cycles_per_s" in b:
        a["fp32_over_fp64"] = a["fwd_adj_cycles_per_s"] / b["fwd_adj_cycles_per_s"]
    return out


def accuracy_study_line(dev, M=12, shift=1, radii=(1, 2, 3), tiles=(6, 12, 16), inflation=1.1):
    """Eq. 18's RMSE over M filter cycles (FP32, enkfmc_filter_run) on one set of
    synthetic inputs for each localisation radius r and sub-domain tile (square,
    in grid cells), the shape of the paper's radius and processor-count studies;
    with the RMSE of the unassimilated background; forecast inflation 1.1."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import WORKLOADS, make_cycle_inputs

    base = WORKLOADS["study_96x48x3x2+1_n60"]
    ci = make_cycle_inputs(base, M, shift, np.float32)  # r and the tile change no input
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ys, Zs, R, xr = put(ci.ys), put(ci.Zs), put(ci.R), put(ci.truths)
    rows = []
    for r in radii:
        for tile in tiles:
            w = base.with_(r=r, sub_lon=tile, sub_lat=tile)
            h = B.Handle.from_workload(w, precision=B.FP32)
            try:
                h.set_observations(ci.obs_idx)
                Xb = put(ci.Xb0)
                T = torch.empty((w.n, h.info.pmax), device=dev)
                D = torch.empty(w.n, device=dev)
                Xa = torch.empty_like(Xb)
                sq = torch.zeros(M, dtype=torch.float64, device=dev)
                h.filter_run(Xb, ys, Zs, R, xr, T, D, Xa, M, shift, sq, inflation)
                code, _ = h.get_status()
                s = sq.cpu().numpy()
                rows.append({"r": r, "tile": tile, "subdomains": h.info.nsub,
                             "rmse_eq18": float(np.sqrt(s.sum() / M)),
                             "rmse_last_per_component": float(np.sqrt(s[-1] / w.n)),
                             "status": B.STATUS.get(code, code)})
            finally:
                h.close()
    e_b = ci.Xb0.astype(np.float64).mean(axis=0) - ci.truths[0].astype(np.float64)
    return {"workload": base.name, "assimilation_times": M, "precision": "fp32",
            "inflation": inflation, "rmse_background": float(np.sqrt(e_b @ e_b)), "runs": rows}


T127_WORKLOAD = "t127_384x192x29_n96_r3"


def t127_line(args, dev, steps=2):
    """The T127-shaped scale case (384 x 192 x 29, n = 2,138,112, N = 96, r = 3,
    ridge where p >= N - 1): one analysis cycle in the mixed-precision default
    (FP32, the rows with 2p > N in double precision, double-precision blocks
    where the single-precision factorisation fails or refines too slowly, four
    refinement steps) against the plain FP32 form (ENKFMC_FLAG_PLAIN_FP32 with
    no refinement), each with its accuracy against the FP64 oracle on sampled
    rows and sub-domains (oracle values from the host cores)."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import WORKLOADS, make_inputs

    w = WORKLOADS[T127_WORKLOAD]
    inp = make_inputs(w, np.float32)
    out = {"workload": w.name, "n": w.n, "N": w.N, "r": w.r}
    ref = tempfile.mktemp(suffix=".npz")
    ncores = args.cpu_workers or os.cpu_count() or 1
    out["oracle_reference"] = run_cpu_sample(w.name, "fp32", 60, 1, ncores, ref)
    forms = (("mixed", 0), ("plain_fp32", B.FLAG_PLAIN_FP32 | B.FLAG_NO_SOLVE_REFINEMENT))
    for key, flags in forms:
        stream = torch.cuda.Stream(device=dev)
        res = {"flags": flags}
        h = None
        try:
            h = B.Handle.from_workload(w, precision=B.FP32, stream=stream.cuda_stream,
                                       flags=flags)
            h.set_observations(inp.obs_idx)
            put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            Xb, y, R, Z = put(inp.Xb), put(inp.y), put(inp.R), put(inp.Z)
            T = torch.empty((w.n, h.info.pmax), device=dev)
            D = torch.empty(w.n, device=dev)
            Xa = torch.empty_like(Xb)

            def cycle():
                h.estimate(Xb, T, D)
                h.assemble(Xb, T, D, R)
                h.analyze(Xb, y, R, Z, Xa)

            ms = _time_steps(cycle, 1, steps, stream)
            code, info = h.get_status()
            res.update({"cycles_per_s": 1e3 / ms, "ms_per_cycle": ms,
                        "status": B.STATUS.get(code, code), "status_info": info,
                        "fp64_rows": bool(h.info.fp64_rows), "refine_steps": h.info.refine_steps,
                        "fp64_blocks": h.fp64_blocks(), "blocks": h.info.nblock,
                        "workspace_gb": h.info.workspace_bytes / 1e9})
            if os.path.exists(ref):
                res["accuracy"] = accuracy_report(w, ref, inp.Xb, T.cpu().numpy(),
                                                  D.cpu().numpy(), Xa.cpu().numpy(), h)
        except Exception as exc:  # report the failure of one form, keep the other
            res["error"] = f"{type(exc).__name__}: {exc}"
        finally:
            if h is not None:
                h.close()
        out[key] = res
    if os.path.exists(ref):
        os.unlink(ref)
    a, b = out.get("mixed", {}), out.get("plain_fp32", {})
    if "cycles_per_s" in a and "cycles_per_s" in b:
        out["mixed_over_plain"] = a["cycles_per_s"] / b["cycles_per_s"]
    return out


def cycling_line(w, dev, M=12, shift=1, inflation=1.1):
    """Filter cycling (Algorithm 1) on workload w in FP32: M assimilation times,
    the forecast operator advecting every field by `shift` cells per step, the
    nature run advected the same way (perfect model), enkfmc_filter_run (cycle 0
    eager, then one captured CUDA graph per cycle); cycles/s over the whole call
    (capture included) and Eq. 18's RMSE, beside the RMSE of the initial
    background mean.  The forecast inflates the ensemble about its mean by
    `inflation` (the advection alone has no model error)."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import make_cycle_inputs

    ci = make_cycle_inputs(w, M, shift, np.float32)
    stream = torch.cuda.Stream(device=dev)
    h = B.Handle.from_workload(w, precision=B.FP32, stream=stream.cuda_stream)
    try:
        h.set_observations(ci.obs_idx)
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        Xb0, ys, Zs, R, xr = put(ci.Xb0), put(ci.ys), put(ci.Zs), put(ci.R), put(ci.truths)
        T = torch.empty((w.n, h.info.pmax), device=dev)
        D = torch.empty(w.n, device=dev)
        Xb, Xa = torch.empty_like(Xb0), torch.empty_like(Xb0)
        sq = torch.zeros(M, dtype=torch.float64, device=dev)
        Xb.copy_(Xb0)
        torch.cuda.synchronize()
        h.filter_run(Xb, ys, Zs, R, xr, T, D, Xa, M, shift, sq, inflation)  # set-up and warm-up
        h.check("cycling warm-up")
        with torch.cuda.stream(stream):
            Xb.copy_(Xb0)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.filter_run(Xb, ys, Zs, R, xr, T, D, Xa, M, shift, sq, inflation)
        e1.record(stream)
        torch.cuda.synchronize()
        h.check("cycling")
        ms = e0.elapsed_time(e1)
        s = sq.cpu().numpy()
        e_b = (ci.Xb0.astype(np.float64).mean(axis=0) - ci.truths[0].astype(np.float64))
        return {"workload": w.name, "precision": "fp32", "assimilation_times": M,
                "shift_cells_per_step": shift, "inflation": inflation,
                "value": M * 1e3 / ms, "unit": "cycles/s",
                "ms_per_cycle": ms / M, "rmse_eq18": float(np.sqrt(s.sum() / M)),
                "rmse_background": float(np.sqrt(e_b @ e_b)),
                "rmse_per_time_per_component": [float(np.sqrt(x / w.n)) for x in s],
                "note": "RMSE of Eq. 18 over the analysis-mean errors of the M times"}
    finally:
        h.close()


def dual_line(w, dev, fracs=(0.04, 0.10), steps=5):
    """The dual form (enkfmc_analyze_dual, Eq. 12-13) against the primal form
    (enkfmc_assemble + enkfmc_analyze) on workload w in FP32, for sparse
    observation networks (the fraction of observed components in `fracs`): both
    from the same enkfmc_estimate, cycles/s of estimate + analysis by CUDA events,
    the dual form's per-kind split, and the largest per-variable difference of
    the two analyses (max |Xa_dual - Xa_primal| / max |Xa_primal|), and the
    number of blocks the primal form factored in double precision.  Where the
    dual form reports a status (ENOTSPD: a block's R + Z^T D Z is not positive
    definite in the arithmetic) the line gives that status and the primal
    form's rate."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import make_inputs

    out = []
    for frac in fracs:
        wf = w.with_(obs_frac=frac)
        inp = make_inputs(wf, np.float32)
        stream = torch.cuda.Stream(device=dev)
        h = B.Handle.from_workload(wf, precision=B.FP32, stream=stream.cuda_stream)
        try:
            h.set_observations(inp.obs_idx)
            with torch.cuda.stream(stream):
                put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                Xb, y, R, Z = put(inp.Xb), put(inp.y), put(inp.R), put(inp.Z)
                T = torch.empty((wf.n, h.info.pmax), device=dev)
                D = torch.empty(wf.n, device=dev)
                Xp, Xd = torch.empty_like(Xb), torch.empty_like(Xb)

            def primal():
                h.estimate(Xb, T, D)
                h.assemble(Xb, T, D, R)
                h.analyze(Xb, y, R, Z, Xp)

            def dual():
                h.estimate(Xb, T, D)
                h.analyze_dual(Xb, T, D, y, R, Z, Xd)

            ms_p = _time_steps(primal, 2, steps, stream)
            h.check("primal form")
            nfb = h.fp64_blocks()
            ms_d = _time_steps(dual, 2, steps, stream)
            code, info = h.get_status()
            if code:  # the dual form does not apply to this problem (reported, not timed)
                out.append({"workload": wf.name, "obs_frac": frac, "m": int(inp.y.size),
                            "primal_fp64_blocks": nfb, "primal_cycles_per_s": 1e3 / ms_p,
                            "primal_ms": ms_p, "dual_status": B.STATUS.get(code, code),
                            "dual_status_block": info})
                continue
            h.profile(True)
            h.profile_read()
            _time_steps(dual, 0, 2, stream)
            prof = h.profile_read()
            h.profile(False)
            primal()
            dual()
            torch.cuda.synchronize()
            h.check("dual form")
            # non-finite values are counted, not folded into the maximum
            nonfinite = {"primal": int((~torch.isfinite(Xp)).sum()),
                         "dual": int((~torch.isfinite(Xd)).sum())}
            diff = 0.0
            for v in range(wf.nvar):
                a = wf.var_offset(v)
                e = a + wf.var_levels(v) * wf.nlat * wf.nlon
                ref = Xp[:, a:e]
                rv = float((Xd[:, a:e] - ref).abs().max() / ref.abs().max())
                diff = rv if rv != rv else max(diff, rv)  # a NaN stays NaN
                if diff != diff:
                    break
            out.append({"workload": wf.name, "obs_frac": frac, "m": int(inp.y.size),
                        "primal_fp64_blocks": nfb,
                        "primal_cycles_per_s": 1e3 / ms_p, "dual_cycles_per_s": 1e3 / ms_d,
                        "primal_ms": ms_p, "dual_ms": ms_d, "dual_speedup": ms_p / ms_d,
                        "max_rel_diff_vs_primal": diff if diff == diff else "nan",
                        "nonfinite": nonfinite,
                        "kernels_ms_per_step": {k: v[1] / 2 for k, v in prof.items() if v[0]}})
        finally:
            h.close()
    return out


def batch_line(args, dev):
    """The 256 independent problems of uneven size (grids 24 x 12 to 96 x 48,
    1-7 levels, 1-5 variables, N 20-120, r 1-4, seeds 3000 + i), FP32, each on
    its own handle with the autotuner's settings (from the tuning cache; the
    library defaults for shapes it lacks), one CUDA graph replay per cycle of
    all of them.  Also the same cycle run eagerly, instance after instance, on
    one stream."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import autotune, binding as B
    from synthetic import make_inputs
    from synthetic.workloads import batch_instances

    ws = batch_instances()
    cache = autotune.load_cache(args.tuning)
    tuned0 = len(cache)
    # with --tune: the shapes with the most work first (the members times the
    # stencil slots times the components), up to --tune-max of them
    work = lambda w: w.N * w.n * (2 * w.r + 1) ** 2 * min(3, w.nlev)
    to_tune = set(sorted(range(len(ws)), key=lambda i: -work(ws[i]))[:args.tune_max])
    stream = torch.cuda.current_stream(dev)
    insts = []
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    for iw, w in enumerate(ws):
        inp = make_inputs(w, np.float32)
        Xb, y, R, Z = put(inp.Xb), put(inp.y), put(inp.R), put(inp.Z)
        choice = cache.get(autotune.shape_key(w, B.FP32))
        mk = lambda c: B.Handle.from_workload(w, precision=B.FP32, stream=stream.cuda_stream,
                                              flags=c["flags"] if c else 0)
        h = mk(choice)
        T = torch.empty((w.n, h.info.pmax), device=dev)
        D = torch.empty(w.n, device=dev)
        Xa = torch.empty_like(Xb)
        if choice is None and args.tune and iw in to_tune:
            choice = autotune.tune(w, inp.obs_idx, (Xb, T, D, y, R, Z, Xa), cache=cache)
            if choice["flags"] != h.problem.flags:
                h.close()
                h = mk(choice)
        if choice:
            autotune.apply(h, choice)
        h.set_observations(inp.obs_idx)
        insts.append((h, (Xb, T, D, y, R, Z, Xa)))
    if args.tune and len(cache) > tuned0:
        autotune.save_cache(cache, args.tuning)
    batch = B.Batch([h for h, _ in insts], nstreams=8, stream=stream.cuda_stream)
    for i, (h, (Xb, T, D, y, R, Z, Xa)) in enumerate(insts):
        batch.bind(i, Xb, T, D, y, R, Z, Xa)
    batch.capture()
    st, _ = batch.status()
    ms = _time_steps(batch.run, 1, 3, stream)
    st2, _ = batch.status()

    def eager():
        for h, (Xb, T, D, y, R, Z, Xa) in insts:
            h.estimate(Xb, T, D)
            h.assemble(Xb, T, D, R)
            h.analyze(Xb, y, R, Z, Xa)

    ms_eager = _time_steps(eager, 0, 1, stream)
    nfb = sum(h.fp64_blocks() for h, _ in insts)
    n_tc = sum(1 for h, _ in insts if not (h.problem.flags & B.FLAG_SIMT_BAND))
    batch.close()
    for h, _ in insts:
        h.close()
    return {"instances": len(ws), "components": int(sum(w.n for w in ws)),
            "members_x_components": int(sum(w.n * w.N for w in ws)),
            "value": 1e3 / ms, "unit": "cycles/s (all instances)", "ms_per_cycle": ms,
            "instances_per_s": len(ws) * 1e3 / ms, "eager_ms_per_cycle": ms_eager,
            "graph_over_eager": ms_eager / ms, "streams": 8,
            "status_nonzero": int((st != 0).sum() + (st2 != 0).sum()),
            "fp64_blocks": int(nfb), "tensor_core_band": n_tc,
            "tuning": (f"{sum(1 for w in ws if autotune.shape_key(w, B.FP32) in cache)} of "
                       f"{len(ws)} shapes from the tuning cache"),
            "instance_list": [w.name for w in ws]}


def plain_fp64_line(w, inp, value, dev):
    """The plain FP64 form of the headline workload, same inputs."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    stream = torch.cuda.Stream(device=dev)
    h = B.Handle.from_workload(w, precision=B.FP64, stream=stream.cuda_stream)
    h.set_observations(inp.obs_idx)
    with torch.cuda.stream(stream):
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev, torch.float64)
        Xb, y, R, Z = put(inp.Xb), put(inp.y), put(inp.R), put(inp.Z)
        T = torch.empty((w.n, h.info.pmax), device=dev, dtype=torch.float64)
        D = torch.empty(w.n, device=dev, dtype=torch.float64)
        Xa = torch.empty_like(Xb)

    def step64():
        h.estimate(Xb, T, D)
        h.assemble(Xb, T, D, R)
        h.analyze(Xb, y, R, Z, Xa)

    ms = _time_steps(step64, 1, 3, stream)
    h.check("fp64 steps")
    h.close()
    return {"workload": w.name, "value": 1e3 / ms, "unit": "cycles/s", "ms_per_step": ms,
            "fp32_over_fp64": value / (1e3 / ms)}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import WORKLOADS, make_inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    w = rank_workload(WORKLOADS[args.workload], rank)
    precision = B.FP64 if args.precision == "fp64" else B.FP32
    npdt = np.float64 if precision == B.FP64 else np.float32
    tdt = torch.float64 if precision == B.FP64 else torch.float32
    esize = 8 if precision == B.FP64 else 4
    inp = make_inputs(w, npdt)
    stream = torch.cuda.Stream(device=dev)
    h = B.Handle.from_workload(w, precision=precision, stream=stream.cuda_stream)
    h.set_observations(inp.obs_idx)
    with torch.cuda.stream(stream):
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev, tdt)
        Xb, y, R, Z = put(inp.Xb), put(inp.y), put(inp.R), put(inp.Z)
        T = torch.empty((w.n, h.info.pmax), device=dev, dtype=tdt)
        D = torch.empty(w.n, device=dev, dtype=tdt)
        Xa = torch.empty_like(Xb)
    stream.synchronize()

    def step():
        h.estimate(Xb, T, D)
        h.assemble(Xb, T, D, R)
        h.analyze(Xb, y, R, Z, Xa)

    for _ in range(args.warmup):
        step()
    h.check("warm-up")
    h.profile(False)
    h.profile_read()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    counts = h.profile_read(kernels=True)            # kernels launched in the timed steps
    h.check("timed steps")
    t_max = slowest_rank(ms, world, dev)
    value = job_rate(args.steps, world, t_max / 1e3)

    # second timed pass with the per-kernel events on: split, roofline, path fraction
    h.profile(True)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.profile_steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof = h.profile_read()
    h.profile(False)
    ms_prof = p0.elapsed_time(p1) / args.profile_steps
    peaks, peak_src = _peaks()
    work = h.work_per_launch()
    sm_max = (clocks or {}).get("sm_max_mhz")
    roof = roofline(prof, work, peaks, peak_src, sm_max, precision == B.FP32, args.workload,
                    args.precision, sm_count)
    tk = {k for k, on in (("bandchol", h.info.tc_chol), ("bandsolve", h.info.tc_solve)) if on}
    path = path_roofline(prof, work, peaks, sm_max, precision == B.FP32, sm_count,
                         args.profile_steps, tk)
    roof["path_frac"] = path["path_frac"]
    roof["timed_region"] = (f"{args.profile_steps} steps after the headline steps, per-kernel "
                            f"events on ({ms_prof:.2f} ms per step)")

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hXb, hy, hR, hZ = pin(inp.Xb), pin(inp.y), pin(inp.R), pin(inp.Z)
        hXa = torch.empty_like(hXb).pin_memory()
        h.cycle_host(hXb, hy, hR, hZ, hXa)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.cycle_host(hXb, hy, hR, hZ, hXa)
        t_e2e = slowest_rank(time.perf_counter() - t0, world, dev)
        m = inp.y.size
        e2e = {"value": job_rate(args.e2e_steps, world, t_e2e), "unit": "cycles/s",
               "h2d_bytes_per_step": esize * (w.N * w.n + 2 * m + w.N * m),
               "d2h_bytes_per_step": esize * w.N * w.n,
               "api": "enkfmc_cycle_host"}

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        step()
        h.check("accuracy step")
        torch.cuda.synchronize()
        ref = tempfile.mktemp(suffix=".npz")
        cpu = cpu_baseline(args, out=ref)
        if os.path.exists(ref):
            accuracy = accuracy_report(w, ref, inp.Xb, T.cpu().numpy(), D.cpu().numpy(),
                                       Xa.cpu().numpy(), h)
            os.unlink(ref)
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            extras = side_measurements(args, w, inp, value, dev)
        except Exception as exc:  # a side line must not hide the headline number
            extras = {"side_measurements_error": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "cycles/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if precision == B.FP64 else "f32", "data": "synthetic",
               "config": workload_config(args, w, world),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(sum(v[1] for v in counts.values())),
               "clocks": clocks, "sm_count": sm_count, "accuracy": accuracy,
               "path_roofline": path,
               "kernels_ms_per_step": {k: v[1] / args.profile_steps for k, v in prof.items()}}
        out.update(extras)
        print(json.dumps(out))
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.t127_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"t127": t127_line(args, torch.device("cuda", 0))}))
        return
    if args.batch_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"batch": batch_line(args, torch.device("cuda", 0))}))
        return
    if args.dual_only:
        import torch

        from synthetic import WORKLOADS
        torch.cuda.set_device(0)
        print(json.dumps({"dual": dual_line(WORKLOADS[args.workload],
                                            torch.device("cuda", 0))}))
        return
    if args.fwd_adj_only:
        import numpy as np
        import torch

        from paper_1606_00807_gb300 import binding as B
        from synthetic import WORKLOADS, make_inputs
        torch.cuda.set_device(0)
        w = WORKLOADS[args.workload]
        line = fwd_adj_line(args, w, make_inputs(w, np.float32), torch.device("cuda", 0),
                            np.float32, B.FP32, torch.float32)
        print(json.dumps({"fwd_adj_fp32": line}))
        return
    if args.cpu_sample:
        cpu_sample_main(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
