"""Reverse-mode derivative of the EnKF-MC analysis (test infrastructure, FP64).

Only the tests, the smoke check and the benchmark's CPU leg use this module.

For a scalar loss L(X^a) the gradient with respect to the background ensemble,
the observations and the observation-error variances is propagated backwards
through every step of the analysis as the paper defines it: the interior
write-back (Eq. 10), the sub-domain solve (Eq. 11, Algorithm 3), the assembly
A = T^T D^-1 T + H^T R^-1 H (Eq. 8, Eq. 11), the modified Cholesky regressions
(Eq. 1-2) and the anomalies (Eq. 5), sub-domain by sub-domain (Algorithm 2).

Per sub-domain k, with W = dL/dX^a on the interior rows (0 on the boundary):
  Lambda = A^-1 W                  (A symmetric)
  Abar   = -Lambda dX^T            (dX = A^-1 rhs)
  rows j: a_j = (T Lambda)_j, b_j = (T dX)_j
     betabar_q = (<a_j, dX_q> + <b_j, Lambda_q>) / D_j   (from Tbar = D^-1 T (Abar + Abar^T))
     Dbar_j    = <a_j, b_j> / D_j^2                      (from the diagonal of T Abar T^T)
  then through e = u - U_P^T beta, beta = (G + lambda I)^-1 g, g = U_P u,
  G = U_P U_P^T, lambda = c tr(G)/p:
     ebar = 2 Dbar e / (N - 1); betabar -= U_P ebar; v = (G + lambda I)^-1 betabar
     f = ebar + U_P^T v;  Ubar_P += v e^T - beta f^T - kappa U_P;  Ubar_j += f
     with kappa = 2 (c/p) v.beta when the ridge is active
  observations o in the extended set (component c):
     ybar_o += sum_i Lambda_ci / R_o
     Rbar_o += (<Lambda_c, dX_c> - <Lambda_c, Delta_o>) / R_o^2
               + <Lambda_c, Z_o> / (2 R_o sqrt(R_o))
     Xbbar_c -= Lambda_c / R_o
Finally Xbbar += dL/dX^a + Ubar - mean_members(Ubar) (the anomaly projection).
"""
from __future__ import annotations

import numpy as np

from .enkfmc import (Grid, anomalies, local_system, perturbed_observations, solve_spd,
                     subdomains)


def _regression_parts(U, j, P, ridge_c):
    """beta, e, D, G + lambda I and lambda of one regression (Eq. 1-2)."""
    N = U.shape[1]
    u = U[j]
    p = len(P)
    if p == 0:
        return np.zeros(0), u.copy(), float(u @ u) / (N - 1), np.zeros((0, 0)), 0.0
    UP = U[np.asarray(P, dtype=np.int64)]
    G = UP @ UP.T
    lam = ridge_c * np.trace(G) / p if (p >= N - 1 and ridge_c > 0) else 0.0
    M = G + lam * np.eye(p)
    beta = np.linalg.solve(M, UP @ u)
    e = u - UP.T @ beta
    return beta, e, float(e @ e) / (N - 1), M, lam


def analysis_with_gradient(w, Xb_mm, y, R, Z_mm, obs_idx, Xa_bar_mm, only=None):
    """X^a and the gradients (Xb_bar [N][n], y_bar [m], R_bar [m]) of a loss whose
    gradient with respect to X^a is Xa_bar (member-major arrays).

    With `only` (sub-domain indices) the other sub-domains are skipped.  A
    sub-domain whose interior rows of Xa_bar are all zero has Lambda = 0, so it
    adds nothing to the gradients; skipping it is then exact.  X^a is returned
    as NaN outside the analysed interiors."""
    grid = Grid.from_workload(w)
    sds = subdomains(grid, w.sub_lon, w.sub_lat)
    Xb = np.asarray(Xb_mm, dtype=np.float64).T
    Z = np.asarray(Z_mm, dtype=np.float64).T
    y = np.asarray(y, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    Wbar = np.asarray(Xa_bar_mm, dtype=np.float64).T
    N = Xb.shape[1]
    U = anomalies(Xb)
    Ys = perturbed_observations(y, R, Z)
    Xa = Xb.copy() if only is None else np.full_like(Xb, np.nan)
    Xb_bar = Wbar.copy()
    y_bar = np.zeros_like(y)
    R_bar = np.zeros_like(R)
    U_bar = np.zeros_like(U)
    for sd in sds:
        if only is not None and sd.index not in only:
            continue
        A, rhs, T, D, o_loc = local_system(grid, sd, U, Xb, Ys, R, obs_idx, w.ridge_c)
        dX = solve_spd(A, rhs)
        pos = {int(q): i for i, q in enumerate(sd.ext)}
        rows = np.array([pos[int(q)] for q in sd.interior])
        Xa[sd.interior] = Xb[sd.interior] + dX[rows]
        W = np.zeros_like(dX)
        W[rows] = Wbar[sd.interior]
        Lam = solve_spd(A, W)
        # observation terms (rhs, Y^s and the H^T R^-1 H part of A)
        for o in o_loc:
            c = pos[int(obs_idx[o])]
            Ro = R[o]
            Delta = Ys[o] - Xb[int(obs_idx[o])]
            y_bar[o] += Lam[c].sum() / Ro
            R_bar[o] += (Lam[c] @ dX[c] - Lam[c] @ Delta) / Ro ** 2 \
                + (Lam[c] @ Z[o]) / (2.0 * Ro * np.sqrt(Ro))
            Xb_bar[int(obs_idx[o])] -= Lam[c] / Ro
        # regression instances of the extended set
        a = T @ Lam
        b = T @ dX
        inside = set(int(q) for q in sd.ext)
        for i, j in enumerate(sd.ext):
            j = int(j)
            P = [q for q in grid.predecessors(j) if q in inside]
            beta, e, Dj, M, lam = _regression_parts(U, j, P, w.ridge_c)
            Ppos = [pos[q] for q in P]
            Dbar = float(a[i] @ b[i]) / Dj ** 2
            ebar = 2.0 * Dbar * e / (N - 1)
            f = ebar.copy()
            if P:
                UP = U[np.asarray(P, dtype=np.int64)]
                betabar = (dX[Ppos] @ a[i] + Lam[Ppos] @ b[i]) / Dj
                betabar = betabar - UP @ ebar
                v = np.linalg.solve(M, betabar)
                f = f + UP.T @ v
                kappa = 2.0 * (w.ridge_c / len(P)) * float(v @ beta) if lam > 0 else 0.0
                U_bar[np.asarray(P, dtype=np.int64)] += np.outer(v, e) - np.outer(beta, f) \
                    - kappa * UP
            U_bar[j] += f
    Xb_bar += U_bar - U_bar.mean(axis=1, keepdims=True)
    return Xa.T, Xb_bar.T, y_bar, R_bar


def loss_mean_analysis(Xa_mm, x_ref):
    """L = 1/2 |mean_members(X^a) - x_ref|^2 and dL/dX^a (member-major)."""
    Xa = np.asarray(Xa_mm, dtype=np.float64)
    N = Xa.shape[0]
    r = Xa.mean(axis=0) - np.asarray(x_ref, dtype=np.float64)
    return 0.5 * float(r @ r), np.repeat((r / N)[None, :], N, axis=0)


def loss_and_gradient(w, Xb_mm, y, R, Z_mm, obs_idx, x_ref):
    """L = 1/2 |mean(X^a) - x_ref|^2 and its gradients w.r.t. X^b, y and diag(R)."""
    from .enkfmc import assimilate
    Xa = assimilate(w, Xb_mm, y, R, Z_mm, obs_idx)
    L, Xa_bar = loss_mean_analysis(Xa, x_ref)
    _, Xb_bar, y_bar, R_bar = analysis_with_gradient(w, Xb_mm, y, R, Z_mm, obs_idx, Xa_bar)
    return L, Xb_bar, y_bar, R_bar
