"""Seeded inputs of a filter-cycling experiment (perfect model).

The nature run: the truth of make_inputs moves `shift` cells eastward along
every latitude circle per assimilation time (the advection that the filter's
forecast operator applies to the members).  At time k the observations are
y_k = truth_k[obs] + sqrt(R) e_k with their own seeded standard normals, and
the perturbed observations draw their own Z_k.  Time 0 reuses make_inputs'
observations and perturbations, and the initial ensemble is make_inputs'.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .fields import make_inputs
from .philox import normal_stream
from .workloads import Workload

_STREAM_CYCLE_NOISE = 5000  # + k
_STREAM_CYCLE_Z = 6000      # + k


@dataclass
class CycleInputs:
    Xb0: np.ndarray     # [N][n] initial background ensemble
    truths: np.ndarray  # [M][n] reference state at each assimilation time
    ys: np.ndarray      # [M][m] observations
    Zs: np.ndarray      # [M][N][m] standard normals of the perturbed observations
    R: np.ndarray       # [m] observation-error variances
    obs_idx: np.ndarray  # [m] observed components (the same at every time)


def nature_run(w: Workload, truth0: np.ndarray, M: int, shift: int) -> np.ndarray:
    """[M][n]: the truth advected by `shift` cells per time (periodic longitude)."""
    planes = w.nvar_3d * w.nlev + w.nvar_2d
    out = np.empty((M, w.n), dtype=np.float64)
    t = np.asarray(truth0, dtype=np.float64).reshape(planes, w.nlat, w.nlon)
    for k in range(M):
        out[k] = t.reshape(-1)
        t = np.roll(t, shift, axis=2)
    return out


def make_cycle_inputs(w: Workload, M: int, shift: int, dtype=np.float64) -> CycleInputs:
    inp = make_inputs(w, np.float64)
    truths = nature_run(w, inp.truth, M, shift)
    m = inp.obs_idx.size
    ys = np.empty((M, m))
    Zs = np.empty((M, w.N, m))
    ys[0], Zs[0] = inp.y, inp.Z
    for k in range(1, M):
        ys[k] = truths[k][inp.obs_idx] + np.sqrt(inp.R) * normal_stream(
            w.seed, _STREAM_CYCLE_NOISE + k, m)
        Zs[k] = normal_stream(w.seed, _STREAM_CYCLE_Z + k, w.N * m).reshape(w.N, m)
    c = lambda a: np.ascontiguousarray(a, dtype=dtype)
    return CycleInputs(c(inp.Xb), c(truths), c(ys), c(Zs), c(inp.R), inp.obs_idx)
