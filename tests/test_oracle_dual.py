"""Pins of the oracle's per-sub-domain dual form (Eq. 12-13).

The dual increment X~ V^T (R + V V^T)^-1 (Y^s - H X^b), T X~ = D^1/2, V = H X~,
equals the primal one (T^T D^-1 T + H^T R^-1 H)^-1 H^T R^-1 (Y^s - H X^b) by the
Sherman-Morrison-Woodbury identity; the primal sub-domain analysis is pinned on
its own (test_oracle_pins.py).  Here: a hand case with a closed form, the
identity on several decompositions (sparse and denser networks, ridge rows, a
wrapped seam, ragged tiles), and the limiting cases.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import oracle.enkfmc as OE
from synthetic import WORKLOADS, make_inputs


def test_dual_increment_hand_case():
    """Two components, T = [[1, 0], [-b, 1]], D = (d1, d2), the second observed:
    B = T^-1 D T^-T = [[d1, b d1], [b d1, b^2 d1 + d2]], and the increment is
    B[:, 1] a / (R + B[1, 1]) for the innovation a."""
    b, d1, d2, R, a = 0.5, 2.0, 1.0, 0.5, 3.0
    T = np.array([[1.0, 0.0], [-b, 1.0]])
    dX = O.dual_increment(T, np.array([d1, d2]), [1], np.array([R]), np.array([[a]]))
    B11 = b * b * d1 + d2
    expect = np.array([b * d1, B11]) * a / (R + B11)      # [1.5, 2.25]
    assert np.allclose(dX[:, 0], expect, rtol=0, atol=1e-15)
    # observing the first component instead: B[:, 0] a / (R + d1)
    dX0 = O.dual_increment(sp.csr_matrix(T), np.array([d1, d2]), [0], np.array([R]),
                           np.array([[a, -a]]))
    assert np.allclose(dX0, np.outer([d1, b * d1], [a, -a]) / (R + d1), rtol=0, atol=1e-15)


def test_dual_increment_requires_lower_triangular_order():
    T = np.array([[1.0, 0.3], [0.0, 1.0]])                 # an upper entry: wrong order
    with pytest.raises(AssertionError):
        O.dual_increment(T, np.ones(2), [0], np.ones(1), np.ones((1, 1)))


@pytest.mark.parametrize("name,frac,kw", [
    ("small_40x30x2x2+1_n48_r2", 0.1, {}),     # ragged tiles, seam, poles, 3 variables
    ("small_40x30x2x2+1_n48_r2", 0.5, {}),     # denser network
    ("small_36x24x2x1_n24_r3_ridge", 0.1, {}), # ridge rows (p >= N - 1)
    ("small_28x20x3x1_n32_r1", 0.3, {}),
    ("small_40x30x2x2+1_n48_r2", 0.15, dict(nlon=16, sub_lon=11)),  # a box of 15 of 16 longitudes
    ("small_40x30x2x2+1_n48_r2", 0.15, dict(lon_periodic=False)),   # no seam
])
def test_dual_analysis_equals_primal(name, frac, kw):
    w = WORKLOADS[name].with_(obs_frac=frac, **kw)
    inp = make_inputs(w)
    only = list(range(0, 12, 2))
    Xp = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, only=only)
    Xd = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, only=only, form="dual")
    done = ~np.isnan(Xp[0])
    assert done.sum() > 0 and np.array_equal(done, ~np.isnan(Xd[0]))
    dp, dd = Xp[:, done] - inp.Xb[:, done], Xd[:, done] - inp.Xb[:, done]
    assert np.abs(dp).max() > 0
    # FP64 rounding of the two routes, amplified by the primal system's condition
    # number (up to ~1e8 with ridge rows); a wrong term or operand moves it by O(1)
    assert O.rel_err(dd, dp) < 1e-7


def test_dual_limiting_cases():
    """No observation in reach: no increment; R -> infinity: X^a -> X^b."""
    w = WORKLOADS["small_28x20x3x1_n32_r1"].with_(obs_frac=0.2)
    inp = make_inputs(w)
    empty = np.zeros(0, dtype=inp.obs_idx.dtype)
    Xa = O.assimilate(w, inp.Xb, inp.y[:0], inp.R[:0], inp.Z[:, :0], empty, form="dual")
    assert np.array_equal(Xa, inp.Xb)
    # (unperturbed observations: the perturbations scale with sqrt(R))
    Xa = O.assimilate(w, inp.Xb, inp.y, inp.R * 1e12, np.zeros_like(inp.Z), inp.obs_idx,
                      form="dual")
    assert np.abs(Xa - inp.Xb).max() < 1e-8 * np.abs(inp.Xb).max()


def test_dual_pins_catch_planted_mistakes():
    """Plausible slips in the dual increment (D left out, T^-1 where T^-T belongs,
    R left out of the observation system) each move the result on a sub-domain
    far beyond the tolerance of the Woodbury pin: the pin would catch them."""
    import scipy.linalg as sla
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"].with_(obs_frac=0.1)
    inp = make_inputs(w)
    g = O.Grid.from_workload(w)
    sd = O.subdomains(g, w.sub_lon, w.sub_lat)[5]
    Xb = inp.Xb.T
    U = O.anomalies(Xb)
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    T, D = O.local_estimate(g, sd, U, w.ridge_c)
    pos = {int(q): i for i, q in enumerate(sd.ext)}
    o_loc = [o for o, c in enumerate(inp.obs_idx) if int(c) in pos]
    hrows = [pos[int(inp.obs_idx[o])] for o in o_loc]
    R = inp.R[o_loc]
    innov = Ys[o_loc] - Xb[sd.ext[hrows]]
    A, rhs, _, _, _ = O.local_system(g, sd, U, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
    primal = OE.solve_spd(A, rhs)
    good = O.dual_increment(T, D, hrows, R, innov)
    assert O.rel_err(good, primal) < 1e-7
    Td = T.toarray()

    def variant(no_d=False, wrong_side=False, no_r=False):
        Dm = np.ones_like(D) if no_d else D
        Xt = sla.solve_triangular(Td.T if wrong_side else Td, np.diag(np.sqrt(Dm)),
                                  lower=not wrong_side, unit_diagonal=True)
        V = Xt[np.asarray(hrows)]
        S = V @ V.T + (0 if no_r else np.diag(R))
        return Xt @ (V.T @ np.linalg.lstsq(S, innov, rcond=None)[0])

    for kw in (dict(no_d=True), dict(wrong_side=True), dict(no_r=True)):
        assert O.rel_err(variant(**kw), primal) > 1e-3, kw


def test_pcg_reaches_the_direct_solve():
    """The preconditioned CG primal solve (M = T^T D^-1 T) converges to the direct
    sub-domain solve of Eq. 11."""
    w = WORKLOADS["small_28x20x3x1_n32_r1"].with_(obs_frac=0.3)
    inp = make_inputs(w)
    g = O.Grid.from_workload(w)
    sd = O.subdomains(g, w.sub_lon, w.sub_lat)[3]
    Xb = inp.Xb.T
    U = O.anomalies(Xb)
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    A, rhs, T, D, _ = O.local_system(g, sd, U, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
    direct = OE.solve_spd(A, rhs[:, :4])
    x, its = OE.pcg_solve(A, rhs[:, :4], T, D, tol=1e-10)
    assert O.rel_err(x, direct) < 1e-7
    assert all(0 < k < 10000 for k in its)
