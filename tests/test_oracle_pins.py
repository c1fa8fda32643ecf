"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
predecessor sets, a brute-force distance enumeration, the inverse sample
covariance (full radius, N > n), the textbook LDL^T factor, SVD least squares,
the Kalman gain form (Eq. 14) and the dual form (Eq. 12-13) of the analysis,
and limiting cases.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from synthetic import WORKLOADS, Workload, make_inputs, normal_stream, philox4x32_10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(**kw):
    kw.setdefault("vert_reach", 1)
    kw.setdefault("lon_periodic", True)
    return O.Grid(kw["nlon"], kw["nlat"], kw["nlev"], kw["nvar_3d"], kw["nvar_2d"], kw["r"],
                  kw["vert_reach"], kw["lon_periodic"])


def _ensemble(n, N, seed, corr=0.6):
    """Correlated Gaussian samples n x N (AR(1) along the label) for pins."""
    z = normal_stream(seed, 7, n * N).reshape(n, N)
    x = np.empty_like(z)
    x[0] = z[0]
    for i in range(1, n):
        x[i] = corr * x[i - 1] + np.sqrt(1 - corr ** 2) * z[i]
    return x


def test_philox_known_answers():
    """Random123 known-answer vectors for Philox4x32-10."""
    cases = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
             ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
             ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
              (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for c, k, want in cases:
        got = philox4x32_10(*[np.uint64(x) for x in c], *[np.uint64(x) for x in k])
        assert tuple(int(x) for x in got) == want


def test_predecessors_hand_fixture():
    """Predecessor sets derived by hand from the local-box rule (Section 2.2-2.3)."""
    d = json.load(open(os.path.join(GOLDEN, "predecessors_hand.json")))
    for case in d["cases"]:
        g = _grid(**case["grid"])
        for j, want in case["rows"].items():
            assert g.predecessors(int(j)) == sorted(want), (case["grid"], j)


@pytest.mark.parametrize("shape", [(7, 5, 2, 1, 1, 1), (6, 4, 3, 1, 0, 2), (3, 4, 1, 2, 0, 2),
                                   (9, 6, 1, 1, 1, 3), (5, 5, 2, 1, 0, 1)])
@pytest.mark.parametrize("periodic", [True, False])
def test_predecessors_bruteforce(shape, periodic):
    """Pattern of T against an O(n^2) enumeration of the distance definition:
    q precedes j iff same variable, |dk| <= 1, max(|dlat|, d_lon) <= r, q < j,
    with d_lon the ring distance when longitude wraps."""
    nlon, nlat, nlev, n3, n2, r = shape
    g = O.Grid(nlon, nlat, nlev, n3, n2, r, 1, periodic)
    C = [g.coords(j) for j in range(g.n)]
    for j in range(g.n):
        vj, kj, aj, oj = C[j]
        want = []
        for q in range(j):
            vq, kq, aq, oq = C[q]
            dl = abs(oq - oj)
            if periodic:
                dl = min(dl, nlon - dl)
            if vq == vj and abs(kq - kj) <= 1 and max(abs(aq - aj), dl) <= r:
                want.append(q)
        assert g.predecessors(j) == want


def test_anomalies_hand_case_and_numpy_covariance():
    """Eq. 5: U = X - mean(X) 1^T.  A hand case, zero row sums over members, and the
    sample covariance U U^T / (N - 1) against numpy's own (independently centred)
    np.cov; a mean taken over components instead of members, or no centring, fails."""
    X = np.array([[1.0, 2.0, 3.0, 6.0], [4.0, 4.0, 4.0, 4.0], [-2.0, 0.0, 2.0, 8.0]])
    U = O.anomalies(X)
    want = np.array([[-2.0, -1.0, 0.0, 3.0], [0.0, 0.0, 0.0, 0.0], [-4.0, -2.0, 0.0, 6.0]])
    assert np.array_equal(U, want)
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    Xb = make_inputs(w).Xb.T                       # n x N
    U = O.anomalies(Xb)
    assert np.abs(U.sum(axis=1)).max() < 1e-12 * np.abs(Xb).max() * w.N
    sub = slice(0, 400)
    S = U[sub] @ U[sub].T / (w.N - 1)
    C = np.cov(Xb[sub])                            # rows are variables, columns samples
    assert np.allclose(S, C, rtol=1e-11, atol=1e-13 * np.abs(C).max())


def test_perturbed_observations_scale_is_sqrt_R():
    """Y^s = y + sqrt(R) z (Section 2.3, Algorithm 1): hand values, and the sample
    variance of Y^s - y over many standard normals equals R (not sqrt R, not R^2)."""
    Ys = O.perturbed_observations(np.array([1.0, -2.0]), np.array([4.0, 0.25]),
                                  np.array([[1.5, -1.0], [2.0, 4.0]]))
    assert np.array_equal(Ys, np.array([[4.0, -1.0], [-1.0, 0.0]]))
    R = np.array([0.01, 4.0, 9.0])
    Z = normal_stream(42, 3, 3 * 200000).reshape(3, 200000)
    d = O.perturbed_observations(np.array([5.0, -1.0, 0.0]), R, Z) - np.array([[5.0], [-1.0], [0.0]])
    var = d.var(axis=1, ddof=1)
    assert np.allclose(var, R, rtol=0.02)


def test_full_radius_reproduces_inverse_sample_covariance():
    """With every earlier component a predecessor and N > n, T^T D^-1 T equals the
    inverse of S = U U^T / (N - 1) (Eq. 1-3 and Eq. 8 with S = U), and T^-1 D T^-T = S."""
    g = O.Grid(4, 3, 1, 1, 0, r=4)           # radius covers the whole grid
    n, N = g.n, 40
    X = _ensemble(n, N, 11)
    U = O.anomalies(X)
    T, D = O.estimate(g, U, ridge_c=0.0)
    S = U @ U.T / (N - 1)
    Binv = (T.T @ np.diag(1.0 / D) @ T)
    assert np.allclose(np.asarray(Binv), np.linalg.inv(S), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.inv(S)).max())
    assert np.allclose(O.b_hat_dense(T, D), S, rtol=1e-10, atol=1e-12)


def test_full_radius_matches_textbook_ldl():
    """T^-1 is the unit lower factor and D the diagonal of S = L D L^T (Cholesky of S
    with its diagonal scaled out), the classical modified Cholesky identity."""
    g = O.Grid(3, 3, 2, 1, 0, r=3, vert_reach=1)
    n, N = g.n, 50
    U = O.anomalies(_ensemble(n, N, 12, corr=0.3))
    T, D = O.estimate(g, U, ridge_c=0.0)
    S = U @ U.T / (N - 1)
    C = np.linalg.cholesky(S)
    Lu = C / np.diag(C)[None, :]
    Tinv = sla.solve_triangular(T.toarray(), np.eye(n), lower=True, unit_diagonal=True)
    assert np.allclose(Tinv, Lu, atol=1e-10)
    assert np.allclose(D, np.diag(C) ** 2, rtol=1e-10)


def test_rows_match_svd_least_squares():
    """Each T row is minus the least-squares coefficients of u_j on U_P (SVD route,
    not the normal equations) and D_j the residual sum of squares over N - 1."""
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    g = O.Grid.from_workload(w)
    inp = make_inputs(w)
    U = O.anomalies(inp.Xb.T)
    rows = list(range(0, g.n, 97)) + [g.n - 1, w.nlon - 1, 2 * w.nlon - 1]
    rows = [j for j in rows if len(g.predecessors(j)) < w.N - 1]      # full-rank Gram
    assert len(rows) > 20
    for j, P, beta, d in O.estimate_rows(g, U, rows, ridge_c=0.0):
        if not P:
            assert d == pytest.approx(np.var(U[j], ddof=1), rel=1e-12)
            continue
        A = U[P].T
        sol, *_ = np.linalg.lstsq(A, U[j], rcond=None)
        res = U[j] - A @ sol
        assert np.allclose(beta, sol, rtol=1e-8, atol=1e-9 * np.abs(sol).max())
        assert d == pytest.approx(res @ res / (w.N - 1), rel=1e-9)


def test_ridge_rows_match_augmented_least_squares():
    """Where p >= N - 1 the ridge regression equals least squares on the
    augmented system [U_P^T; sqrt(lambda) I] beta ~ [u_j; 0], lambda = c tr(G)/p."""
    w = WORKLOADS["small_36x24x2x1_n24_r3_ridge"]
    g = O.Grid.from_workload(w)
    U = O.anomalies(make_inputs(w).Xb.T)
    seen = 0
    for j, P, beta, d in O.estimate_rows(g, U, range(0, g.n, 53), ridge_c=w.ridge_c):
        p = len(P)
        if p < w.N - 1:
            continue
        seen += 1
        UP = U[P]
        lam = w.ridge_c * np.trace(UP @ UP.T) / p
        A = np.vstack([UP.T, np.sqrt(lam) * np.eye(p)])
        b = np.concatenate([U[j], np.zeros(p)])
        sol, *_ = np.linalg.lstsq(A, b, rcond=None)
        assert np.allclose(beta, sol, rtol=1e-7, atol=1e-8 * np.abs(sol).max())
        e = U[j] - UP.T @ sol
        assert d == pytest.approx(e @ e / (w.N - 1), rel=1e-8)
        assert d > 0
    assert seen > 10


def test_structure_unit_lower_positive_D():
    w = WORKLOADS["tiny_32x16_n20_r2"]
    g = O.Grid.from_workload(w)
    U = O.anomalies(make_inputs(w).Xb.T)
    T, D = O.estimate(g, U, w.ridge_c)
    Td = T.toarray()
    assert np.all(np.diag(Td) == 1.0)
    assert np.count_nonzero(np.triu(Td, 1)) == 0
    assert np.all(D > 0)
    # p = 0 row: the first component has D = var(u).
    assert D[0] == pytest.approx(np.var(U[0], ddof=1), rel=1e-12)
    # the pattern of T is the predecessor rule
    rowptr, col = O.t_pattern_csr(g)
    for j in range(g.n):
        nz = np.nonzero(Td[j, :j])[0]
        assert list(nz) == list(col[rowptr[j]:rowptr[j + 1]])
    # largest predecessor count at r = 2 on one level: 2 rows of 5 + 2 left + 2 wrapped
    assert max(np.diff(rowptr)) == 14


def _one_domain(w: Workload) -> Workload:
    return w.with_(sub_lon=w.nlon, sub_lat=w.nlat)


@pytest.mark.parametrize("name,N", [("tiny_32x16_n20_r2", 20), ("small_28x20x3x1_n32_r1", 48)])
def test_primal_equals_gain_and_dual_forms(name, N):
    """One sub-domain covering the grid: the primal increment (Eq. 11) equals the
    gain form x_a = x_b + B H^T (H B H^T + R)^-1 (y^s - H x_b) with B = T^-1 D T^-T
    (Eq. 9, Eq. 14) and the dual form (Eq. 12-13)."""
    # N well above p keeps B = T^-1 D T^-T conditioned enough for the dense forms
    w = _one_domain(WORKLOADS[name]).with_(N=N)
    g = O.Grid.from_workload(w)
    inp = make_inputs(w)
    Xb = inp.Xb.T
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    assert len(sds) == 1 and len(sds[0].ext) == g.n
    Xa = O.analysis(g, sds, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
    U = O.anomalies(Xb)
    T, D = O.estimate(g, U, w.ridge_c)
    Xg = O.gain_form_analysis(Xb, Ys, inp.R, inp.obs_idx, O.b_hat_dense(T, D))
    Xd = O.dual_form_analysis(T, D, Xb, Ys, inp.R, inp.obs_idx)
    assert O.rel_err(Xa - Xb, Xg - Xb) < 1e-8
    assert O.rel_err(Xa - Xb, Xd - Xb) < 1e-8


def test_subdomain_increment_equals_local_gain_form():
    """With a decomposition, each sub-domain's interior analysis equals the gain form
    with its local B_k = T_k^-1 D_k T_k^-T and the observations of its extended set."""
    w = WORKLOADS["tiny_32x16_n20_r2"]
    g = O.Grid.from_workload(w)
    inp = make_inputs(w)
    Xb = inp.Xb.T
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    U = O.anomalies(Xb)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    Xa = O.analysis(g, sds, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
    for sd in sds[::3]:
        T, D = O.local_estimate(g, sd, U, w.ridge_c)
        pos = {int(q): i for i, q in enumerate(sd.ext)}
        o_loc = [o for o, c in enumerate(inp.obs_idx) if int(c) in pos]
        Xl = O.gain_form_analysis(Xb[sd.ext], Ys[o_loc], inp.R[o_loc],
                                  [pos[int(inp.obs_idx[o])] for o in o_loc], O.b_hat_dense(T, D))
        rows = [pos[int(q)] for q in sd.interior]
        assert O.rel_err(Xa[sd.interior] - Xb[sd.interior], Xl[rows] - Xb[sd.interior]) < 1e-8


def test_subdomain_tiling_and_halo():
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    # 40 = 12+12+12+4 and 30 = 12+12+6: a ragged tile in both directions
    assert len(sds) == 4 * 3
    interiors = np.concatenate([sd.interior for sd in sds])
    assert np.array_equal(np.sort(interiors), np.arange(g.n))       # disjoint cover
    for sd in sds:
        ext = set(int(q) for q in sd.ext)
        assert set(int(q) for q in sd.interior) <= ext
        # interior rows keep every predecessor: local rows equal global rows (Algorithm 3)
        for j in sd.interior[:: max(1, len(sd.interior) // 50)]:
            assert all(q in ext for q in g.predecessors(int(j)))
    # the first tile wraps across the longitude seam and is clipped at the pole
    first = sds[0]
    lons = sorted({g.coords(int(q))[3] for q in first.ext})
    lats = sorted({g.coords(int(q))[2] for q in first.ext})
    assert lons == [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 38, 39]
    assert lats == list(range(0, 14))


def test_special_cases_no_obs_and_huge_R():
    """No observation in reach => no increment; R -> infinity => X^a -> X^b."""
    w = WORKLOADS["tiny_32x16_n20_r2"]
    g = O.Grid.from_workload(w)
    inp = make_inputs(w)
    Xb = inp.Xb.T
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    # observations only in the first tile's interior rows 0-3: far tiles get no increment
    keep = np.array([o for o, c in enumerate(inp.obs_idx) if g.coords(int(c))[2] < 4 and g.coords(int(c))[3] < 4])
    Ys = O.perturbed_observations(inp.y[keep], inp.R[keep], inp.Z.T[keep])
    Xa = O.analysis(g, sds, Xb, Ys, inp.R[keep], inp.obs_idx[keep], w.ridge_c)
    far = sds[len(sds) - 3]
    assert np.array_equal(Xa[far.interior], Xb[far.interior])
    assert np.abs(Xa[sds[0].interior] - Xb[sds[0].interior]).max() > 0
    Rbig = inp.R * 1e12
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    Xa = O.analysis(g, sds, Xb, Ys, Rbig, inp.obs_idx, w.ridge_c)
    assert np.abs(Xa - Xb).max() < 1e-8 * np.abs(Xb).max()
    # Z = 0 gives unperturbed observations
    assert np.array_equal(O.perturbed_observations(inp.y, inp.R, np.zeros_like(inp.Z.T)),
                          np.repeat(inp.y[:, None], w.N, axis=1))


def test_analysis_reduces_error_against_truth():
    """Sanity of the synthetic set-up: the analysis mean is closer to the truth."""
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w)
    Xa = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    eb = np.sqrt(np.mean((inp.Xb.mean(0) - inp.truth) ** 2))
    ea = np.sqrt(np.mean((Xa.mean(0) - inp.truth) ** 2))
    assert ea < 0.8 * eb
