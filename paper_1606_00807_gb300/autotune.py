"""Launch autotuner: per problem shape, time candidate launch settings of one
analysis cycle through the C ABI and keep the fastest, cached as JSON.

The settings change how the library launches its kernels, never what they
compute: the band path (the rank-32 panel updates of the band Cholesky and
solves on the tensor cores, or on the CUDA cores: ENKFMC_FLAG_SIMT_BAND) and
the grid cap of the regressions' grid-stride launch (CTAs per SM,
ENKFMC_TUNE_REGRESS_CTAS_PER_SM).  Timing uses CUDA events on the handle's
stream around whole cycles (estimate, assemble, analyze) after a warm-up
cycle.  The cache maps shape_key(...) to the chosen settings and the timings
of every candidate; a shape found in the cache is not timed again.
"""
from __future__ import annotations

import json
import os

from . import binding as B

BAND_PATHS = (0, B.FLAG_SIMT_BAND)
REGRESS_CAPS = (16, 32, 64)


def shape_key(w, precision) -> str:
    """Cache key of a problem shape: grid, variables, radius, members, tile, precision."""
    return (f"{w.nlon}x{w.nlat}x{w.nlev}x{w.nvar_3d}+{w.nvar_2d}_r{w.r}_vr{w.vert_reach}"
            f"_n{w.N}_t{w.sub_lon}x{w.sub_lat}_p{int(bool(w.lon_periodic))}_{precision}")


def load_cache(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(cache, path):
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_cycles(torch, h, bufs, reps):
    Xb, T, D, y, R, Z, Xa = bufs
    stream = torch.cuda.current_stream()

    def cycle():
        h.estimate(Xb, T, D)
        h.assemble(Xb, T, D, R)
        h.analyze(Xb, y, R, Z, Xa)

    cycle()
    h.check("autotune warm-up")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        cycle()
    e1.record(stream)
    torch.cuda.synchronize()
    h.check("autotune cycles")
    return e0.elapsed_time(e1) / reps


def tune(w, obs_idx, bufs, precision=B.FP32, reps=2, cache=None, flags=0):
    """Settings for workload w: {"flags", "regress_cap", "ms", "timings"}.

    obs_idx: the observed labels (host); bufs = (Xb, T, D, y, R, Z, Xa) device
    tensors of one instance of w, T and D shaped for its handle.  Looks the
    shape up in `cache` (a dict) first and stores the result there."""
    import torch
    key = shape_key(w, precision)
    if cache is not None and key in cache:
        return cache[key]
    timings = {}
    best = None
    paths = BAND_PATHS if precision == B.FP32 else (0,)
    stream = torch.cuda.current_stream().cuda_stream
    for path in paths:
        h = B.Handle.from_workload(w, precision=precision, stream=stream, flags=flags | path)
        try:
            h.set_observations(obs_idx)
            for cap in REGRESS_CAPS:
                h.set_tuning(B.TUNE_REGRESS_CTAS_PER_SM, cap)
                try:
                    ms = _time_cycles(torch, h, bufs, reps)
                except B.EnkfmcError as exc:   # a candidate that fails is not chosen
                    timings[f"band{path}_cap{cap}"] = f"failed: {exc}"
                    continue
                timings[f"band{path}_cap{cap}"] = ms
                if best is None or ms < best["ms"]:
                    best = {"flags": flags | path, "regress_cap": cap, "ms": ms}
        finally:
            h.close()
    if best is None:
        raise RuntimeError(f"no launch setting of {key} completed: {timings}")
    best["timings"] = timings
    if cache is not None:
        cache[key] = best
    return best


def apply(handle, choice):
    """Apply a tuned choice's runtime knobs to a handle created with its flags."""
    handle.set_tuning(B.TUNE_REGRESS_CTAS_PER_SM, int(choice["regress_cap"]))
