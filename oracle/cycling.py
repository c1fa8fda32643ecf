"""Filter cycling (Algorithm 1) in FP64 (test infrastructure).

Algorithm 1 alternates the analysis step with the model step of every member.
The model here is the synthetic forecast operator of the cycling experiment:
every field moves `shift` cells eastward along its latitude circle per step
(periodic longitude).  Eq. 18 measures the analysis accuracy over the M
assimilation times: RMSE = sqrt( (1/M) sum_k |x_ref_k - x_a_k|^2 ), with x_a_k
the analysis ensemble mean at time k (the reading taken: the paper's x^a_k is
the analysis state, which for an ensemble filter is its mean).  The forecast
may inflate the ensemble about its mean by a factor rho (multiplicative
covariance inflation): the shift alone has no model error, so a cycled
ensemble's spread would only shrink.
"""
from __future__ import annotations

import numpy as np

from .enkfmc import assimilate


def forecast_shift(w, X_mm: np.ndarray, shift: int, inflation: float = 1.0) -> np.ndarray:
    """Member-major [nvec][n] states, each field advected by `shift` cells:
    out[..., x] = in[..., x - shift] along longitude (periodic), after
    X = mean + inflation (X - mean) about the mean of the nvec vectors."""
    X = np.asarray(X_mm, dtype=np.float64)
    if inflation != 1.0:
        mean = X.mean(axis=0)
        X = mean + inflation * (X - mean)
    nvec = X.shape[0]
    planes = w.n // (w.nlat * w.nlon)
    out = np.empty_like(X)
    for v in range(nvec):
        f = X[v].reshape(planes, w.nlat, w.nlon)
        g = np.empty_like(f)
        for x in range(w.nlon):
            g[:, :, (x + shift) % w.nlon] = f[:, :, x]
        out[v] = g.reshape(-1)
    return out


def ensemble_sqerr(Xa_mm: np.ndarray, xref: np.ndarray) -> float:
    """|mean_m Xa[m] - xref|^2 (the summand of Eq. 18)."""
    e = np.asarray(Xa_mm, dtype=np.float64).mean(axis=0) - np.asarray(xref, dtype=np.float64)
    return float(e @ e)


def rmse_eq18(sqerrs) -> float:
    """Eq. 18 from the per-time squared errors |x_ref_k - x_a_k|^2."""
    s = np.asarray(sqerrs, dtype=np.float64)
    return float(np.sqrt(s.sum() / s.size))


def filter_cycles(w, Xb0, ys, Zs, R, xrefs, obs_idx, shift, inflation=1.0):
    """M cycles of Algorithm 1: analysis of the background with y_k, Z_k, the
    squared error of its mean against x_ref_k, then the forecast of every
    member.  Returns (per-time squared errors [M], last analysis [N][n],
    background after the last forecast [N][n])."""
    Xb = np.asarray(Xb0, dtype=np.float64)
    sq = []
    Xa = Xb
    for k in range(len(xrefs)):
        Xa = assimilate(w, Xb, ys[k], R, Zs[k], obs_idx)
        sq.append(ensemble_sqerr(Xa, xrefs[k]))
        Xb = forecast_shift(w, Xa, shift, inflation)
    return np.array(sq), Xa, Xb
