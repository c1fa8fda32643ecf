#!/usr/bin/env python3
"""Throughput of the EnKF-MC analysis step on GB300: analysis cycles per second.

One step = one analysis cycle of the whole hot path on one synthetic ensemble
already resident in HBM: enkfmc_estimate (anomalies + the regressions of every
component), enkfmc_assemble (boundary re-estimation, band assembly, banded
Cholesky of every sub-domain block) and enkfmc_analyze (right-hand sides,
N-member band solves, interior write-back).  Workload: the T63-shaped state
(192 x 96 x (7 levels x 4 variables + 1), n = 534,528), N = 80 members,
r = 2, 12 x 12 sub-domains with an r-wide boundary, 50% of the components
observed; FP32 by default.  Inputs are larger than L2 (X^b alone is 171 MB
in FP32), so no flush is needed between steps.

Printed: one JSON line with the contract keys, the roofline of the dominant
kernel (timed live with CUDA events on the library's stream), the end-to-end
rate through enkfmc_cycle_host from pinned host buffers, the SM clocks seen
during the timed region, and the FP64 oracle timed on a bounded sample on the
host cores.  Multi-GPU (torchrun): every rank runs an independent problem (its
own seed); value = cycles of all ranks / slowest rank's time.

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
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture of its current version on the named workload and
# precision (the capture commands are in profiles/); a kernel without one
# reports null.
TRAFFIC_PER_LAUNCH = {("regress", "t63_192x96x29_n80_r2", "fp32"): 724.3e6}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-FP64 and forward+adjoint side measurements")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-rows", type=int, default=1000)
    ap.add_argument("--sample-subdomains", type=int, default=3)
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
# CPU oracle timing (bounded sample), used by cpu_baseline and --impl reference
# ----------------------------------------------------------------------------
def oracle_sample_time(w, inp, nrows, nsub, seed=0):
    """Seconds per full analysis cycle of the FP64 oracle, extrapolated from
    `nrows` global regressions and `nsub` sub-domain analyses."""
    import numpy as np
    import oracle as O
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    rng = np.random.default_rng(seed)
    Xb = inp.Xb.T.astype(np.float64)
    t0 = time.perf_counter()
    U = O.anomalies(Xb)
    t_anom = time.perf_counter() - t0
    rows = rng.choice(g.n, nrows, replace=False)
    t0 = time.perf_counter()
    O.estimate_rows(g, U, rows, w.ridge_c)
    t_row = (time.perf_counter() - t0) / nrows
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    picks = rng.choice(len(sds), nsub, replace=False)
    t0 = time.perf_counter()
    for i in picks:
        O.local_analysis(g, sds[int(i)], U, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
    t_sd = (time.perf_counter() - t0) / nsub
    cycle = t_anom + t_row * g.n + t_sd * len(sds)
    return cycle, f"{nrows} of {g.n} regressions + {nsub} of {len(sds)} sub-domain analyses"


def cpu_sample_main(args):
    """Child process (one thread): time the oracle and print one JSON line."""
    import numpy as np
    from synthetic import WORKLOADS, make_inputs
    w = WORKLOADS[args.workload]
    dt = np.float64 if args.precision == "fp64" else np.float32
    inp = make_inputs(w, dt)
    cycle, sample = oracle_sample_time(w, inp, args.sample_rows, args.sample_subdomains)
    print(json.dumps({"cycle_s": cycle, "sample": sample}))


def cpu_baseline(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", args.workload,
           "--precision", args.precision, "--sample-rows", str(args.sample_rows),
           "--sample-subdomains", str(args.sample_subdomains)]
    p = subprocess.run(cmd, capture_output=True, text=True, env=env)
    if p.returncode != 0:
        return {"error": p.stderr.strip().splitlines()[-1] if p.stderr.strip() else "failed"}
    d = json.loads(p.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / d["cycle_s"], "unit": "cycles/s", "cores": 1, "kind": "oracle",
            "sample": d["sample"] + " (FP64 numpy/scipy oracle, one thread; cycle time "
                      "extrapolated to the full workload)"}


# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def roofline(prof, work, peaks, peak_src, sm_max_mhz, fp32, workload, precision):
    """Roofline of the dominant kernel (largest device time per cycle).

    prof: kernel -> (launches, ms); work: kernel -> (flops, bytes) per launch.
    The bound is the one whose time per launch is larger at its peak: FP32 FMA
    lanes at the maximum SM clock (or FP64 nominal) for flops, the measured
    copy bandwidth for bytes; achieved = the algorithmic work per launch over
    the kernel's average launch time."""
    dom = max(prof, key=lambda k: prof[k][1])
    launches, dom_ms = prof[dom]
    avg_s = dom_ms / max(1, launches) / 1e3
    flops, nbytes = work[dom]
    sm_max = sm_max_mhz or peaks.get("sm_max_mhz", 2070.0)
    if fp32:
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        alu_note = (f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                    f"{sm_max:.0f} MHz")
    else:
        alu_peak = FP64_NOMINAL_TFLOPS
        alu_note = "FP64 nominal 1.25 TFLOP/s"
    t_alu = flops / (alu_peak * 1e12)
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    if t_alu >= t_hbm:
        achieved = flops / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "peak_source": f"derived: {alu_note}"}
    else:
        achieved = nbytes / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peak_src} hbm_gbs"}
    roof["traffic"] = TRAFFIC_PER_LAUNCH.get((dom, workload, precision))
    roof["kernel"] = dom
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["algorithmic_per_launch"] = {"flops": flops, "bytes": nbytes}
    return roof


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
    import numpy as np
    from synthetic import WORKLOADS, make_inputs
    w = WORKLOADS[args.workload]
    inp = make_inputs(w, np.float64 if args.precision == "fp64" else np.float32)
    cyc = []
    sample = ""
    for s in range(args.warmup + args.steps):
        c, sample = oracle_sample_time(w, inp, 200, 1, seed=s)
        if s >= args.warmup:
            cyc.append(c)
    mean_cycle = sum(cyc) / len(cyc)
    value = 1.0 / mean_cycle
    cores = 1
    try:
        import threadpoolctl  # noqa: F401
        cores = max(i["num_threads"] for i in threadpoolctl.threadpool_info()) if \
            threadpoolctl.threadpool_info() else 1
    except Exception:
        cores = os.cpu_count() or 1
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cycles/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean_cycle * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, w, 1),
           "cpu_baseline": {"value": value, "unit": "cycles/s", "cores": cores, "kind": "oracle",
                            "sample": "per step: " + sample + "; cycle time extrapolated"},
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


def fwd_adj_line(wa, ia, dev, npdt, precision, tdt):
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
    h.close()
    return {"workload": wa.name, "precision": "fp32" if precision == B.FP32 else "fp64",
            "fwd_cycles_per_s": 1e3 / ms_f, "fwd_adj_cycles_per_s": 1e3 / ms_fa,
            "fwd_ms": ms_f, "fwd_adj_ms": ms_fa, "adj_over_fwd": (ms_fa - ms_f) / ms_f,
            "kernels_ms_per_step": {k: v[1] / 2 for k, v in prof.items() if v[0]}}


def side_measurements(args, w, inp, value, dev):
    """Side lines of the headline metric, each on its own handle: the plain
    FP64 form of the same workload (cycles/s and the FP32 speed-up over it);
    forward + adjoint (the loss L = 1/2 |mean(X^a) - x_ref|^2, its gradient
    dL/dX^a formed on the device, then enkfmc_analyze_adjoint for X^b, y and
    diag(R)) against the forward analysis alone, on the same workload in FP32
    and at the T63 shape with N = 40 in FP64."""
    import numpy as np
    import torch

    from paper_1606_00807_gb300 import binding as B
    from synthetic import WORKLOADS, make_inputs

    out = {}
    # plain FP64 form, same workload and inputs
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
    del Xb, y, R, Z, T, D, Xa
    out["plain_fp64"] = {"workload": w.name, "value": 1e3 / ms, "unit": "cycles/s",
                         "ms_per_step": ms, "fp32_over_fp64": value / (1e3 / ms)}

    out["fwd_adj_fp32"] = fwd_adj_line(w, inp, dev, np.float32, B.FP32, torch.float32)

    # forward + adjoint, T63 shape with N = 40: p = 37 predecessors from 40
    # members make the Gram matrices nearly singular, so this configuration runs
    # in FP64 (single precision reports EDNONPOS here)
    wa = WORKLOADS["t63_192x96x29_n40_r2"]
    out["fwd_adj"] = fwd_adj_line(wa, make_inputs(wa, np.float64), dev, np.float64, B.FP64,
                                  torch.float64)
    return out


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
    h.profile(True)
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
    prof = h.profile_read()
    h.profile(False)
    h.check("timed steps")
    t_max = slowest_rank(ms, world, dev)
    value = job_rate(args.steps, world, t_max / 1e3)

    # roofline of the dominant kernel
    peaks, peak_src = _peaks()
    roof = roofline(prof, h.work_per_launch(), peaks, peak_src,
                    (clocks or {}).get("sm_max_mhz"), precision == B.FP32, args.workload,
                    args.precision)

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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)
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
               "gpu_launches": int(sum(v[0] for v in prof.values())),
               "clocks": clocks,
               "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()}}
        out.update(extras)
        print(json.dumps(out))
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.cpu_sample:
        cpu_sample_main(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
