"""Seeded synthetic inputs for one assimilation problem.

Fields are separable Gaussian random fields with covariance
    sigma_v^2 * rho^|dk| * exp(-d_lon / L) * exp(-|d_lat| / L),
where d_lon is the periodic (ring) distance when longitude wraps.  A draw
multiplies a standard-normal array by Cholesky factors of the two 1-D
correlation matrices and chains the levels as a first-order autoregression
with coefficient rho.  The exponential of the ring distance is a positive
definite correlation on the circle, so both factors exist.

truth   = one draw
centre  = truth + one draw         (the background the ensemble is built around)
Xb[i]   = centre + one draw, i = 0..N-1, stored member-major [N][n]
obs     = a seeded random subset of components (or every second one)
R       = r_frac * sigma_v^2 of the observed variable
y       = truth[obs] + sqrt(R) * e,   e ~ N(0, 1)
Z       = [N][m] standard normals used for the perturbed observations

Random numbers come from Philox4x32-10 streams (see `philox`).  This module
only makes inputs; it holds none of the filter's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np

from .philox import normal_stream, uint32_stream
from .workloads import Workload

_STREAM_OBS_PICK = 2
_STREAM_OBS_NOISE = 3
_STREAM_Z = 4
_STREAM_TRUTH = 100
_STREAM_CENTRE = 101
_STREAM_MEMBER0 = 1000


@dataclass
class Inputs:
    Xb: np.ndarray        # [N][n] member-major
    y: np.ndarray         # [m]
    R: np.ndarray         # [m] observation-error variances (diagonal of R)
    Z: np.ndarray         # [N][m] standard normals
    obs_idx: np.ndarray   # [m] int32, sorted, unique component labels
    truth: np.ndarray     # [n]

    def astype(self, dtype) -> "Inputs":
        return Inputs(self.Xb.astype(dtype), self.y.astype(dtype), self.R.astype(dtype),
                      self.Z.astype(dtype), self.obs_idx, self.truth.astype(dtype))


@lru_cache(maxsize=16)
def _corr_factor(npts: int, length: float, periodic: bool) -> np.ndarray:
    i = np.arange(npts)
    d = np.abs(i[:, None] - i[None, :]).astype(np.float64)
    if periodic:
        d = np.minimum(d, npts - d)
    return np.linalg.cholesky(np.exp(-d / length))


def variable_of(w: Workload, labels: np.ndarray) -> np.ndarray:
    """Variable index of each component label."""
    bounds = np.array([w.var_offset(v) for v in range(1, w.nvar)] + [w.n], dtype=np.int64)
    return np.searchsorted(bounds, labels, side="right")


def draw_field(w: Workload, stream: int) -> np.ndarray:
    """One Gaussian random field over all n components (label order), float64."""
    llat = _corr_factor(w.nlat, w.corr_len, False)
    llon = _corr_factor(w.nlon, w.corr_len, w.lon_periodic)
    z = normal_stream(w.seed, stream, w.n)
    out = np.empty(w.n, dtype=np.float64)
    a = np.sqrt(max(0.0, 1.0 - w.rho_vert ** 2))
    for v in range(w.nvar):
        nl = w.var_levels(v)
        off = w.var_offset(v)
        zz = z[off:off + nl * w.nlat * w.nlon].reshape(nl, w.nlat, w.nlon)
        f = llat @ zz @ llon.T
        for k in range(1, nl):
            f[k] = w.rho_vert * f[k - 1] + a * f[k]
        out[off:off + f.size] = np.sqrt(w.sigma2[v]) * f.reshape(-1)
    return out


def observation_indices(w: Workload) -> np.ndarray:
    if w.obs == "every2":
        return np.arange(0, w.n, 2, dtype=np.int32)
    if w.obs == "random":
        m = int(round(w.obs_frac * w.n))
        keys = uint32_stream(w.seed, _STREAM_OBS_PICK, w.n)
        pick = np.argsort(keys, kind="stable")[:m]
        return np.sort(pick).astype(np.int32)
    if w.obs == "none":
        return np.zeros(0, dtype=np.int32)
    raise ValueError(f"unknown observation rule {w.obs!r}")


def make_inputs(w: Workload, dtype=np.float64) -> Inputs:
    truth = draw_field(w, _STREAM_TRUTH)
    centre = truth + draw_field(w, _STREAM_CENTRE)
    Xb = np.empty((w.N, w.n), dtype=np.float64)
    for i in range(w.N):
        Xb[i] = centre + draw_field(w, _STREAM_MEMBER0 + i)
    obs_idx = observation_indices(w)
    m = obs_idx.size
    sig2 = np.asarray(w.sigma2, dtype=np.float64)
    R = w.r_frac * sig2[variable_of(w, obs_idx.astype(np.int64))]
    y = truth[obs_idx] + np.sqrt(R) * normal_stream(w.seed, _STREAM_OBS_NOISE, m)
    Z = normal_stream(w.seed, _STREAM_Z, w.N * m).reshape(w.N, m)
    return Inputs(Xb, y, R, Z, obs_idx, truth).astype(dtype)
