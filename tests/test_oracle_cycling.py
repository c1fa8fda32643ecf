"""Pins of the oracle's filter cycling (Algorithm 1 with the synthetic forecast
operator, Eq. 18), against hand-worked values and properties that hold exactly."""
import numpy as np

import oracle as O
from synthetic import WORKLOADS, make_cycle_inputs, make_inputs, nature_run
from synthetic.workloads import Workload


def _line(nlon, nlat=1):
    return Workload(name="line", nlon=nlon, nlat=nlat, nlev=1, nvar_3d=1, nvar_2d=0, r=1, N=2,
                    sub_lon=nlon, sub_lat=nlat, sigma2=(1.0,))


def test_forecast_shift_hand_example():
    w = _line(4)
    X = np.array([[0.0, 1.0, 2.0, 3.0], [10.0, 11.0, 12.0, 13.0]])
    assert np.array_equal(O.forecast_shift(w, X, 1), [[3, 0, 1, 2], [13, 10, 11, 12]])
    assert np.array_equal(O.forecast_shift(w, X, 4), X)           # a full turn
    assert np.array_equal(O.forecast_shift(w, X, -1), O.forecast_shift(w, X, 3))
    w2 = _line(3, nlat=2)                                           # each latitude circle alone
    Y = np.arange(6.0)[None]
    assert np.array_equal(O.forecast_shift(w2, Y, 1), [[2, 0, 1, 5, 3, 4]])


def test_forecast_inflation_hand_example_and_moments():
    """Two vectors [0, 2] and [2, 4] (mean [1, 3]) inflated by 2 about their mean
    give [-1, 1] and [3, 5], then shifted by one cell: [1, -1] and [5, 3].  In
    general the mean is kept and the sample variance scales by rho^2."""
    w = _line(2)
    X = np.array([[0.0, 2.0], [2.0, 4.0]])
    assert np.array_equal(O.forecast_shift(w, X, 1, inflation=2.0), [[1, -1], [5, 3]])
    rng = np.random.default_rng(0)
    w5 = _line(5)
    Y = rng.standard_normal((6, 5))
    Z = O.forecast_shift(w5, Y, 0, inflation=1.3)
    assert np.allclose(Z.mean(axis=0), Y.mean(axis=0), rtol=0, atol=1e-14)
    assert np.allclose(Z.var(axis=0), 1.3 ** 2 * Y.var(axis=0), rtol=1e-12)


def test_sqerr_and_eq18_hand_examples():
    assert O.ensemble_sqerr(np.array([[1.0, 2.0], [3.0, 4.0]]), np.zeros(2)) == 13.0
    assert np.isclose(O.rmse_eq18([1.0, 3.0]), np.sqrt(2.0))
    assert O.rmse_eq18([4.0]) == 2.0


def test_nature_run_is_the_forecast_of_the_truth():
    """The generator's nature run (np.roll) and the oracle's forecast operator
    (an explicit loop) agree: truth_{k+1} = M(truth_k)."""
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    t0 = make_inputs(w).truth
    tr = nature_run(w, t0, 4, 3)
    for k in range(3):
        assert np.array_equal(O.forecast_shift(w, tr[k][None], 3)[0], tr[k + 1])


def test_cycling_without_observations_keeps_the_initial_error():
    """With no observations every analysis returns its background, and the
    forecast is a permutation applied to the truth as well, so every time has
    the initial squared error |mean(Xb0) - truth0|^2 and Eq. 18 gives its root."""
    w = WORKLOADS["tiny_32x16_n20_r2"].with_(obs="none")
    M, shift = 4, 2
    ci = make_cycle_inputs(w, M, shift)
    sq, Xa, Xb = O.filter_cycles(w, ci.Xb0, ci.ys, ci.Zs, ci.R, ci.truths, ci.obs_idx, shift)
    e0 = ci.Xb0.mean(axis=0) - ci.truths[0]
    assert np.allclose(sq, e0 @ e0, rtol=1e-12)
    assert np.isclose(O.rmse_eq18(sq), np.sqrt(e0 @ e0))
    assert np.allclose(Xb, O.forecast_shift(w, ci.Xb0, M * shift), rtol=0, atol=1e-12)


def test_cycling_with_observations_beats_the_background():
    """Assimilating half the components each time pulls the mean towards the
    truth: every analysis error is below the initial background error."""
    w = WORKLOADS["tiny_32x16_n20_r2"]
    M, shift = 3, 1
    ci = make_cycle_inputs(w, M, shift)
    sq, _, _ = O.filter_cycles(w, ci.Xb0, ci.ys, ci.Zs, ci.R, ci.truths, ci.obs_idx, shift)
    e0 = ci.Xb0.mean(axis=0) - ci.truths[0]
    assert np.all(sq < e0 @ e0)
