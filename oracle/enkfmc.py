"""EnKF-MC analysis step, written out from the paper in FP64 (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  Matrices follow the paper's orientation: a state ensemble is n x N
(one column per member, Eq. 4), observations are m x N.  Callers holding
member-major [N][n] arrays pass their transposes.

Readings of points the paper leaves open (each one a line of the design notes):
  * var(eps) in Eq. 1-2 is the residual sum of squares over N - 1;
  * component ranges start at 1: a component with no predecessors has
    D = var(u) and an empty T row;
  * predecessors are the neighbours with a smaller label, where neighbours
    share the variable, lie within `vert_reach` levels and within Chebyshev
    distance r on the (lat, periodic lon) grid (Section 2.2, Section 2.3 and
    Fig. 2 describe the local box and the labelling);
  * the regression solves the normal equations by Cholesky (Gram matrix),
    with a ridge lambda = ridge_c * tr(G) / p wherever p >= N - 1;
  * the local update of Algorithm 3 is Eq. 11 (H^T R^-1 applied to the
    innovation);
  * a sub-domain's boundary is r columns wide on every side, clipped at the
    poles and wrapped in longitude; observations inside the boundary enter
    the local system; only interior analyses are kept (Section 3, Eq. 14);
  * Y^s = y 1^T + diag(sqrt(R)) Z with Z an input, not re-centred.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Grid, labels and the localisation rule (Section 2.2, Section 2.3, Fig. 1-2)
# ----------------------------------------------------------------------------
class Grid:
    """Labelled model grid.

    Label of (variable v, level k, latitude j, longitude i) is
    offset(v) + (k * nlat + j) * nlon + i; 3-D variables come first with
    `nlev` levels each, 2-D variables follow with one level.
    """

    def __init__(self, nlon: int, nlat: int, nlev: int, nvar_3d: int, nvar_2d: int, r: int,
                 vert_reach: int = 1, lon_periodic: bool = True):
        self.nlon, self.nlat, self.nlev = nlon, nlat, nlev
        self.nvar_3d, self.nvar_2d = nvar_3d, nvar_2d
        self.r, self.vert_reach, self.lon_periodic = r, vert_reach, bool(lon_periodic)
        self.levels = [nlev] * nvar_3d + [1] * nvar_2d
        self.offsets = [0]
        for nl in self.levels:
            self.offsets.append(self.offsets[-1] + nl * nlat * nlon)
        self.n = self.offsets[-1]

    @classmethod
    def from_workload(cls, w) -> "Grid":
        return cls(w.nlon, w.nlat, w.nlev, w.nvar_3d, w.nvar_2d, w.r, w.vert_reach, w.lon_periodic)

    def coords(self, j: int) -> Tuple[int, int, int, int]:
        v = 0
        while j >= self.offsets[v + 1]:
            v += 1
        rem = j - self.offsets[v]
        k, rem = divmod(rem, self.nlat * self.nlon)
        lat, lon = divmod(rem, self.nlon)
        return v, k, lat, lon

    def label(self, v: int, k: int, lat: int, lon: int) -> int:
        return self.offsets[v] + (k * self.nlat + lat) * self.nlon + lon

    def neighbourhood(self, j: int) -> set:
        """Components other than j in j's local box: same variable, level within
        vert_reach, Chebyshev distance <= r with longitude taken on the ring."""
        v, k, lat, lon = self.coords(j)
        out = set()
        for dk in range(-self.vert_reach, self.vert_reach + 1):
            kk = k + dk
            if not 0 <= kk < self.levels[v]:
                continue
            for dlat in range(-self.r, self.r + 1):
                la = lat + dlat
                if not 0 <= la < self.nlat:
                    continue
                for dlon in range(-self.r, self.r + 1):
                    lo = lon + dlon
                    if self.lon_periodic:
                        lo %= self.nlon
                    elif not 0 <= lo < self.nlon:
                        continue
                    q = self.label(v, kk, la, lo)
                    if q != j:
                        out.add(q)
        return out

    def predecessors(self, j: int) -> List[int]:
        """Neighbours of j that come before j in the labelling (Eq. 1 restricted
        to the local box, Section 2.3), in increasing label order."""
        return sorted(q for q in self.neighbourhood(j) if q < j)


def t_pattern_csr(grid: Grid) -> Tuple[np.ndarray, np.ndarray]:
    """Strictly-lower pattern of T as CSR (rowptr int64 [n+1], colidx int32)."""
    rowptr = np.zeros(grid.n + 1, dtype=np.int64)
    cols: List[int] = []
    for j in range(grid.n):
        p = grid.predecessors(j)
        cols.extend(p)
        rowptr[j + 1] = rowptr[j] + len(p)
    return rowptr, np.asarray(cols, dtype=np.int32)


# ----------------------------------------------------------------------------
# Sub-domains (Section 3, Fig. 3, Eq. 14, Algorithm 2)
# ----------------------------------------------------------------------------
@dataclass
class Subdomain:
    index: int
    lat0: int
    lat1: int
    lon0: int
    lon1: int
    interior: np.ndarray   # sorted labels of the tile's own components
    ext: np.ndarray        # sorted labels of tile + r-wide boundary


def subdomains(grid: Grid, sub_lon: int, sub_lat: int) -> List[Subdomain]:
    """Tile the (lat, lon) plane into sub_lat x sub_lon columns (the last tile
    in each direction may be smaller) and add an r-wide boundary on every side,
    clipped at the poles and wrapped in longitude.  Tiles are numbered
    latitude-major, longitude fastest."""
    r = grid.r
    out = []
    for lat0 in range(0, grid.nlat, sub_lat):
        lat1 = min(grid.nlat, lat0 + sub_lat)
        for lon0 in range(0, grid.nlon, sub_lon):
            lon1 = min(grid.nlon, lon0 + sub_lon)
            lats_in = range(lat0, lat1)
            lons_in = range(lon0, lon1)
            lats_ext = range(max(0, lat0 - r), min(grid.nlat, lat1 + r))
            if grid.lon_periodic:
                width = min(lon1 - lon0 + 2 * r, grid.nlon)
                lons_ext = sorted({(lon0 - r + t) % grid.nlon for t in range(width)})
            else:
                lons_ext = range(max(0, lon0 - r), min(grid.nlon, lon1 + r))
            interior, ext = [], []
            for v in range(len(grid.levels)):
                for k in range(grid.levels[v]):
                    for la in lats_in:
                        for lo in lons_in:
                            interior.append(grid.label(v, k, la, lo))
                    for la in lats_ext:
                        for lo in lons_ext:
                            ext.append(grid.label(v, k, la, lo))
            out.append(Subdomain(len(out), lat0, lat1, lon0, lon1,
                                 np.array(sorted(interior), dtype=np.int64),
                                 np.array(sorted(ext), dtype=np.int64)))
    return out


# ----------------------------------------------------------------------------
# Ensemble statistics (Eq. 5) and perturbed observations (Section 2.3)
# ----------------------------------------------------------------------------
def anomalies(Xb: np.ndarray) -> np.ndarray:
    """U^b = X^b - mean(X^b) 1^T for an n x N ensemble (Eq. 5)."""
    Xb = np.asarray(Xb, dtype=np.float64)
    return Xb - Xb.mean(axis=1, keepdims=True)


def perturbed_observations(y: np.ndarray, R: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Y^s = y 1^T + diag(sqrt(R)) Z, with Z an m x N array of standard normals:
    each column is y plus a draw from N(0, R) (Section 2.3, Algorithm 1)."""
    y = np.asarray(y, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return y[:, None] + np.sqrt(R)[:, None] * np.asarray(Z, dtype=np.float64)


# ----------------------------------------------------------------------------
# Modified Cholesky regressions (Eq. 1-3, Eq. 8)
# ----------------------------------------------------------------------------
def regress(U: np.ndarray, j: int, P: Sequence[int], ridge_c: float) -> Tuple[np.ndarray, float]:
    """Regress the anomalies of component j on those of its predecessors P (Eq. 1).

    Returns (beta, D_j): beta solves (G + lambda I) beta = U_P u_j with the Gram
    matrix G = U_P U_P^T, lambda = ridge_c * tr(G) / p where p >= N - 1 (else 0),
    and D_j = |u_j - U_P^T beta|^2 / (N - 1) is the residual variance (Eq. 2).
    Raises numpy.linalg.LinAlgError when G + lambda I is not positive definite.
    """
    N = U.shape[1]
    uj = U[j]
    p = len(P)
    if p == 0:
        e = uj
        beta = np.zeros(0)
    else:
        UP = U[np.asarray(P, dtype=np.int64)]
        G = UP @ UP.T
        g = UP @ uj
        lam = ridge_c * np.trace(G) / p if (p >= N - 1 and ridge_c > 0) else 0.0
        L = np.linalg.cholesky(G + lam * np.eye(p))
        w = sla.solve_triangular(L, g, lower=True)
        beta = sla.solve_triangular(L.T, w, lower=False)
        e = uj - UP.T @ beta
    return beta, float(e @ e) / (N - 1)


def estimate_rows(grid: Grid, U: np.ndarray, rows: Sequence[int], ridge_c: float,
                  within: np.ndarray | None = None):
    """Rows of T and entries of D for the given components.

    Predecessor sets are the global ones, or their intersection with the label
    set `within` (a sub-domain's extended set, Algorithm 3).  Returns a list of
    (j, P, beta, D_j)."""
    inside = None if within is None else set(int(x) for x in within)
    out = []
    for j in rows:
        j = int(j)
        P = grid.predecessors(j)
        if inside is not None:
            P = [q for q in P if q in inside]
        beta, d = regress(U, j, P, ridge_c)
        out.append((j, P, beta, d))
    return out


def estimate(grid: Grid, U: np.ndarray, ridge_c: float):
    """Global T (unit lower triangular, CSR) and D (Eq. 1-3 with S = U, Eq. 8)."""
    rows, cols, vals = [], [], []
    D = np.zeros(grid.n)
    for j, P, beta, d in estimate_rows(grid, U, range(grid.n), ridge_c):
        rows.append(j); cols.append(j); vals.append(1.0)
        rows.extend([j] * len(P)); cols.extend(P); vals.extend((-beta).tolist())
        D[j] = d
    T = sp.csr_matrix((vals, (rows, cols)), shape=(grid.n, grid.n))
    return T, D


def local_estimate(grid: Grid, sd: Subdomain, U: np.ndarray, ridge_c: float):
    """T_k and D_k on a sub-domain's extended set, from the local samples only
    (Algorithm 3, first step): each predecessor set is cut to the extended set.
    Rows and columns follow the order of `sd.ext`."""
    pos = {int(q): i for i, q in enumerate(sd.ext)}
    ne = len(sd.ext)
    rows, cols, vals = [], [], []
    D = np.zeros(ne)
    for j, P, beta, d in estimate_rows(grid, U, sd.ext, ridge_c, within=sd.ext):
        i = pos[j]
        rows.append(i); cols.append(i); vals.append(1.0)
        for q, b in zip(P, beta):
            rows.append(i); cols.append(pos[q]); vals.append(-b)
        D[i] = d
    return sp.csr_matrix((vals, (rows, cols)), shape=(ne, ne)), D


# ----------------------------------------------------------------------------
# Local analysis (Eq. 10-11, Eq. 14, Algorithms 2-3)
# ----------------------------------------------------------------------------
def local_system(grid: Grid, sd: Subdomain, U: np.ndarray, Xb: np.ndarray, Ys: np.ndarray,
                 R: np.ndarray, obs_idx: np.ndarray, ridge_c: float):
    """A_k = T_k^T D_k^-1 T_k + H_k^T R_k^-1 H_k and rhs_k = H_k^T R_k^-1 (Y^s_k - H_k X^b_k)
    on the extended set (Eq. 8, Eq. 11); H_k selects the observations whose
    component lies in the extended set.  Returns (A, rhs, T, D, local obs ids)."""
    T, D = local_estimate(grid, sd, U, ridge_c)
    ne = len(sd.ext)
    pos = {int(q): i for i, q in enumerate(sd.ext)}
    o_loc = [o for o, c in enumerate(obs_idx) if int(c) in pos]
    H = sp.csr_matrix((np.ones(len(o_loc)), (np.arange(len(o_loc)),
                                              [pos[int(obs_idx[o])] for o in o_loc])),
                      shape=(len(o_loc), ne))
    Rinv = sp.diags(1.0 / np.asarray(R, dtype=np.float64)[o_loc]) if o_loc else sp.csr_matrix((0, 0))
    A = T.T @ sp.diags(1.0 / D) @ T
    if o_loc:
        A = A + H.T @ Rinv @ H
        innov = Ys[o_loc] - H @ Xb[sd.ext]
        rhs = H.T @ (Rinv @ innov)
    else:
        rhs = np.zeros((ne, Xb.shape[1]))
    return sp.csr_matrix(A), np.asarray(rhs), T, D, np.asarray(o_loc, dtype=np.int64)


def solve_spd(A, rhs: np.ndarray) -> np.ndarray:
    """A^-1 rhs for the local SPD system (dense Cholesky when small, sparse LU
    otherwise); either route is the plain definition of the solve in Eq. 11."""
    n = A.shape[0]
    if n <= 3000:
        c = sla.cho_factor(A.toarray(), lower=True)
        return sla.cho_solve(c, rhs)
    lu = spla.splu(sp.csc_matrix(A))
    return lu.solve(np.asarray(rhs, dtype=np.float64))


def local_analysis(grid: Grid, sd: Subdomain, U, Xb, Ys, R, obs_idx, ridge_c):
    """delta X_k = A_k^-1 rhs_k on the extended set (Eq. 11, Algorithm 3)."""
    A, rhs, _, _, _ = local_system(grid, sd, U, Xb, Ys, R, obs_idx, ridge_c)
    return solve_spd(A, rhs)


def dual_increment(T, D: np.ndarray, hrows: Sequence[int], R: np.ndarray,
                   innov: np.ndarray) -> np.ndarray:
    """The dual increment (Eq. 12-13) for one domain: T Xt = D^(1/2) with T unit
    lower triangular, V = H Xt (H selects the rows `hrows`),
    delta X = Xt V^T (R + V V^T)^-1 innov, innov = Y^s - H X^b (m x N)."""
    Td = T.toarray() if sp.issparse(T) else np.asarray(T, dtype=np.float64)
    ne = Td.shape[0]
    if len(hrows) == 0:
        return np.zeros((ne, innov.shape[1]))
    assert not np.any(np.triu(Td, 1)), "T must be lower triangular in the given order"
    Xt = sla.solve_triangular(Td, np.diag(np.sqrt(np.asarray(D, dtype=np.float64))),
                              lower=True, unit_diagonal=True)
    V = Xt[np.asarray(hrows, dtype=np.int64)]
    S = np.diag(np.asarray(R, dtype=np.float64)) + V @ V.T
    return Xt @ (V.T @ np.linalg.solve(S, innov))


def local_dual_analysis(grid: Grid, sd: Subdomain, U, Xb, Ys, R, obs_idx, ridge_c):
    """delta X_k of a sub-domain in the dual form (Eq. 12-13) on its extended set,
    with the same T_k, D_k (Algorithm 3) and local observations as the primal
    form (local_system); T_k is lower triangular in the label order of sd.ext."""
    T, D = local_estimate(grid, sd, U, ridge_c)
    pos = {int(q): i for i, q in enumerate(sd.ext)}
    o_loc = [o for o, c in enumerate(obs_idx) if int(c) in pos]
    hrows = [pos[int(obs_idx[o])] for o in o_loc]
    innov = Ys[o_loc] - Xb[sd.ext[hrows]] if o_loc else np.zeros((0, Xb.shape[1]))
    return dual_increment(T, D, hrows, np.asarray(R, dtype=np.float64)[o_loc], innov)


def pcg_solve(A, rhs: np.ndarray, T, D: np.ndarray, tol: float = 1e-6, maxit: int = 10000):
    """A x = rhs column by column by conjugate gradients preconditioned with
    M = T^T D^-1 T (M^-1 r = T^-1 D T^-T r, two unit-triangular solves), the
    iterative primal solve the paper mentions beside Eq. 11.  Stops when
    |r| <= tol |rhs| per column.  Returns (x, iterations per column)."""
    Tc = sp.csr_matrix(T)
    Tt = sp.csr_matrix(T.T)
    Dv = np.asarray(D, dtype=np.float64)

    def minv(r):
        u = spla.spsolve_triangular(Tt, r, lower=False, unit_diagonal=True)
        return spla.spsolve_triangular(Tc, Dv * u, lower=True, unit_diagonal=True)

    A = sp.csr_matrix(A)
    rhs = np.asarray(rhs, dtype=np.float64)
    X = np.zeros_like(rhs)
    its = []
    for c in range(rhs.shape[1]):
        b = rhs[:, c]
        nb = np.linalg.norm(b)
        x = np.zeros_like(b)
        if nb == 0.0:
            its.append(0)
            continue
        r = b.copy()
        z = minv(r)
        p = z.copy()
        rz = r @ z
        k = 0
        while np.linalg.norm(r) > tol * nb and k < maxit:
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            z = minv(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            k += 1
        X[:, c] = x
        its.append(k)
    return X, its


def analysis(grid: Grid, sds: List[Subdomain], Xb, Ys, R, obs_idx, ridge_c,
             only: Sequence[int] | None = None, form: str = "primal"):
    """Algorithm 2: every sub-domain analyses its extended set independently, the
    boundary is discarded and the interior is written into X^a (Eq. 10).

    Xb is n x N.  With `only`, just those sub-domains are analysed and the
    returned X^a holds NaN elsewhere.  form: "primal" (Eq. 11) or "dual"
    (Eq. 12-13)."""
    Xb = np.asarray(Xb, dtype=np.float64)
    U = anomalies(Xb)
    Xa = np.full_like(Xb, np.nan) if only is not None else Xb.copy()
    local = {"primal": local_analysis, "dual": local_dual_analysis}[form]
    for sd in sds:
        if only is not None and sd.index not in only:
            continue
        dX = local(grid, sd, U, Xb, Ys, R, obs_idx, ridge_c)
        pos = {int(q): i for i, q in enumerate(sd.ext)}
        rows = [pos[int(q)] for q in sd.interior]
        Xa[sd.interior] = Xb[sd.interior] + dX[rows]
    return Xa


def assimilate(w, Xb_mm, y, R, Z_mm, obs_idx, only=None, form: str = "primal"):
    """One analysis from member-major inputs (Xb [N][n], Z [N][m]) for a
    workload-like object with grid, radius, tile and ridge fields; returns
    X^a member-major (form as for analysis)."""
    grid = Grid.from_workload(w)
    sds = subdomains(grid, w.sub_lon, w.sub_lat)
    Ys = perturbed_observations(y, R, np.asarray(Z_mm, dtype=np.float64).T)
    Xa = analysis(grid, sds, np.asarray(Xb_mm, dtype=np.float64).T, Ys, R, obs_idx,
                  w.ridge_c, only=only, form=form)
    return Xa.T


# ----------------------------------------------------------------------------
# Dense forms used to cross-check the primal solve (Eq. 9, Eq. 12-14)
# ----------------------------------------------------------------------------
def b_hat_dense(T, D: np.ndarray) -> np.ndarray:
    """B-hat = T^-1 D T^-T (Eq. 9), dense."""
    Td = T.toarray() if sp.issparse(T) else np.asarray(T)
    Tinv = sla.solve_triangular(Td, np.eye(Td.shape[0]), lower=True, unit_diagonal=True)
    return Tinv @ np.diag(D) @ Tinv.T


def gain_form_analysis(Xb, Ys, R, obs_idx, Bhat) -> np.ndarray:
    """X^a = X^b + B H^T (R + H B H^T)^-1 (Y^s - H X^b) (the Kalman gain form
    of Eq. 14 for one domain); n x N arrays."""
    H = np.zeros((len(obs_idx), Xb.shape[0]))
    H[np.arange(len(obs_idx)), np.asarray(obs_idx)] = 1.0
    S = np.diag(R) + H @ Bhat @ H.T
    return Xb + Bhat @ H.T @ np.linalg.solve(S, Ys - H @ Xb)


def dual_form_analysis(T, D, Xb, Ys, R, obs_idx) -> np.ndarray:
    """Dual increment (Eq. 12-13): T Xt = D^(1/2), V = H Xt,
    delta X = Xt V^T (R + V V^T)^-1 (Y^s - H X^b)."""
    Td = T.toarray() if sp.issparse(T) else np.asarray(T)
    Xt = sla.solve_triangular(Td, np.diag(np.sqrt(D)), lower=True, unit_diagonal=True)
    V = Xt[np.asarray(obs_idx)]
    dX = Xt @ V.T @ np.linalg.solve(np.diag(R) + V @ V.T, Ys - Xb[np.asarray(obs_idx)])
    return Xb + dX


def rel_err(M: np.ndarray, M_ref: np.ndarray) -> float:
    """max |M - M_ref| / max |M_ref| (0 when both vanish)."""
    M = np.asarray(M, dtype=np.float64)
    M_ref = np.asarray(M_ref, dtype=np.float64)
    den = np.max(np.abs(M_ref)) if M_ref.size else 0.0
    num = np.max(np.abs(M - M_ref)) if M_ref.size else 0.0
    return float(num / den) if den > 0 else float(num)
