"""Pins of the oracle's reverse-mode gradient: FP64 central finite differences of
L = 1/2 |mean(X^a) - x_ref|^2 in random directions of X^b, y and diag(R), on a
plain case and on a case where the ridge is active (p >= N - 1)."""
import numpy as np
import pytest

import oracle as O
from oracle.adjoint import analysis_with_gradient, loss_and_gradient, loss_mean_analysis
from synthetic import WORKLOADS, make_inputs


def _loss(w, Xb, y, R, Z, obs_idx, x_ref):
    Xa = O.assimilate(w, Xb, y, R, Z, obs_idx)
    return loss_mean_analysis(Xa, x_ref)[0]


@pytest.mark.parametrize("case", ["plain", "ridge"])
def test_gradient_matches_central_differences(case):
    w = WORKLOADS["tiny_32x16_n20_r2"]
    if case == "ridge":
        w = w.with_(N=12, ridge_c=1e-3, sub_lon=16, sub_lat=8)
    inp = make_inputs(w)
    x_ref = inp.truth
    L, Xb_bar, y_bar, R_bar = loss_and_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx,
                                                x_ref)
    rng = np.random.default_rng(11)
    # directions: X^b, y, and a relative change of diag(R)
    dX = rng.standard_normal(inp.Xb.shape)
    dy = rng.standard_normal(inp.y.shape)
    dR = rng.standard_normal(inp.R.shape) * inp.R
    # the ridge case (N = 12) is ill-conditioned: in the diag(R) direction rounding
    # in L dominates below h ~ 1e-5, so that direction takes a larger step
    # (truncation error ~1e-7 relative); X^b and y keep h = 1e-6
    tol = 1e-6 if case == "plain" else 1e-5
    for name, d, grad in (("Xb", dX, Xb_bar), ("y", dy, y_bar), ("R", dR, R_bar)):
        h = 1e-4 if (case == "ridge" and name == "R") else 1e-6
        args_p = [inp.Xb, inp.y, inp.R]
        args_m = [inp.Xb, inp.y, inp.R]
        k = {"Xb": 0, "y": 1, "R": 2}[name]
        args_p = [a + h * d if i == k else a for i, a in enumerate(args_p)]
        args_m = [a - h * d if i == k else a for i, a in enumerate(args_m)]
        fd = (_loss(w, args_p[0], args_p[1], args_p[2], inp.Z, inp.obs_idx, x_ref)
              - _loss(w, args_m[0], args_m[1], args_m[2], inp.Z, inp.obs_idx, x_ref)) / (2 * h)
        an = float(np.sum(grad * d))
        assert abs(fd - an) <= tol * max(abs(fd), abs(an)) + 1e-10 * abs(L), (name, fd, an)


def test_gradient_of_analysis_is_linear_in_the_output_gradient():
    """The reverse pass is linear in dL/dX^a: gradients for W1 + 2 W2 equal those for
    W1 plus twice those for W2 (checks no term depends on the seed twice)."""
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w)
    rng = np.random.default_rng(3)
    W1 = rng.standard_normal(inp.Xb.shape)
    W2 = rng.standard_normal(inp.Xb.shape)
    g1 = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W1)
    g2 = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W2)
    g3 = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W1 + 2 * W2)
    for a, b, c in zip(g1[1:], g2[1:], g3[1:]):
        assert np.allclose(c, a + 2 * b, rtol=1e-9, atol=1e-12 * np.abs(c).max())
    # and the forward part equals the plain analysis
    Xa = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    assert np.allclose(g1[0], Xa, rtol=0, atol=1e-12 * np.abs(Xa).max())


@pytest.mark.parametrize("name,ridge", [("tiny_32x16_n20_r2", False),
                                        ("small_36x24x2x1_n24_r3_ridge", True)])
def test_regression_residual_normal_equations(name, ridge):
    """The regression residual e = u_j - U_P^T beta of (G + lambda I) beta =
    U_P u_j, G = U_P U_P^T (Eq. 1 with the ridge) satisfies U_P e = lambda beta;
    the GPU adjoint takes <U_qi, ebar> from this instead of a pass over U_P.
    Checked against the oracle's own regressions, rows with and without the
    ridge, to rounding relative to |U_P| |u_j|."""
    from oracle.adjoint import _regression_parts
    w = WORKLOADS[name]
    g = O.Grid.from_workload(w)
    U = O.anomalies(make_inputs(w).Xb.T)
    seen_ridge = seen_plain = 0
    for j in range(0, g.n, 7):
        P = g.predecessors(j)
        if not P:
            continue
        beta, e, _, _, lam = _regression_parts(U, j, P, w.ridge_c)
        UP = U[np.asarray(P, dtype=np.int64)]
        scale = np.abs(UP).sum(axis=1).max() * np.abs(U[j]).max()
        assert np.allclose(UP @ e, lam * beta, rtol=0, atol=1e-11 * scale)
        if lam > 0:
            seen_ridge += 1
            assert np.abs(UP @ e).max() > 1e3 * 1e-11 * scale  # the ridge term is not rounding
        else:
            seen_plain += 1
    assert seen_plain > 5
    if ridge:
        assert seen_ridge > 5


def test_gradient_of_one_subdomain_seed_needs_only_that_subdomain():
    """A seed dL/dX^a that vanishes outside one sub-domain's interior leaves every other
    sub-domain with Lambda = 0: the gradient computed from that sub-domain alone equals
    the full one (the reduction the T63 gradient check on the GPU relies on)."""
    from oracle.adjoint import analysis_with_gradient
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w)
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    k0 = 5
    W = np.zeros((w.N, w.n))
    W[:, sds[k0].interior] = np.random.default_rng(1).standard_normal((w.N, len(sds[k0].interior)))
    full = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W)
    part = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W, only=[k0])
    for a, b in zip(full[1:], part[1:]):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(a).max())
    assert np.allclose(part[0][:, sds[k0].interior], full[0][:, sds[k0].interior])
    assert np.isnan(part[0][:, sds[0].interior]).all()
