"""Filter cycling on the GPU (enkfmc_forecast_shift, enkfmc_ensemble_sqerr,
enkfmc_filter_run) against the FP64 oracle's Algorithm 1 with the same forecast
operator, and the captured-graph replay against the same calls made eagerly.

Tolerances: the forecast is a permutation (bit-exact); the squared error sums
in double precision (1e-12 relative against numpy's sum of the same values).
FP32 cycles: every analysis adds an error near 5e-7, and each next analysis
re-estimates B^-1 from the ensemble it inherits, so an inherited error e
returns as about a e with a > 1; over M = 12 cycles that sums to
e_M = eps (a^M - 1) / (a - 1), 39 eps for a = 1.2 and 1e-4 for a = 1.45
(measured on the 32 x 16 case with N = 20: 3.2e-5 in the ensemble, 7e-6 in the
squared errors).  FP64: 1e-9."""
import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_cycle_inputs

from _harness import per_variable_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _handle(torch, B, w, precision, obs_idx):
    h = B.Handle.from_workload(w, precision=precision,
                               stream=torch.cuda.current_stream().cuda_stream)
    h.set_observations(obs_idx)
    return h


@pytest.mark.parametrize("precision", [0, 1])
def test_forecast_and_sqerr_match_oracle(torch_cuda, precision):
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    dt = np.float64 if precision == 0 else np.float32
    rng = np.random.default_rng(5)
    X = rng.standard_normal((w.N, w.n)).astype(dt)
    xref = rng.standard_normal(w.n).astype(dt)
    h = _handle(torch, B, w, precision, np.zeros(0, np.int64))
    try:
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        for shift in (1, 7, -3, w.nlon):
            h.forecast_shift(Xd, Yd, w.N, shift)
            assert np.array_equal(Yd.cpu().numpy(), O.forecast_shift(w, X, shift).astype(dt)), shift
        for rho in (1.1, 0.9):
            h.forecast_shift(Xd, Yd, w.N, 5, rho)
            ref = O.forecast_shift(w, X, 5, inflation=rho)
            err = np.abs(Yd.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max()
            assert err < (1e-14 if precision == 0 else 2e-7), (rho, err)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        h.ensemble_sqerr(Xd, torch.from_numpy(xref).cuda(), out)
        ref = O.ensemble_sqerr(X.astype(np.float64), xref.astype(np.float64))
        assert abs(out.item() - ref) <= 1e-12 * ref
    finally:
        h.close()


def _inputs_on_device(torch, ci, dt):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    return dev(ci.Xb0), dev(ci.ys), dev(ci.Zs), dev(ci.R), dev(ci.truths)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,inflation", [("tiny_32x16_n20_r2", 1.0),
                                            ("small_48x26x3x1+1_n80_r2", 1.0),
                                            ("small_48x26x3x1+1_n80_r2", 1.1)])
def test_filter_run_matches_oracle(torch_cuda, name, inflation, precision):
    """M = 12 cycles (Eq. 18's twelve assimilation times), shift 1 cell per step,
    with and without covariance inflation in the forecast."""
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS[name]
    M, shift = 12, 1
    dt = torch.float64 if precision == 0 else torch.float32
    ci = make_cycle_inputs(w, M, shift, np.float64 if precision == 0 else np.float32)
    sq_ref, Xa_ref, Xb_ref = O.filter_cycles(w, ci.Xb0, ci.ys, ci.Zs, ci.R, ci.truths,
                                             ci.obs_idx, shift, inflation)
    h = _handle(torch, B, w, precision, ci.obs_idx)
    try:
        Xb, ys, Zs, R, xr = _inputs_on_device(torch, ci, dt)
        T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=dt)
        D = torch.empty(w.n, device="cuda", dtype=dt)
        Xa = torch.empty_like(Xb)
        sq = torch.zeros(M, dtype=torch.float64, device="cuda")
        h.filter_run(Xb, ys, Zs, R, xr, T, D, Xa, M, shift, sq, inflation)
        h.check("filter_run")
        sq = sq.cpu().numpy()
        lab = np.arange(w.n)
        eXa = per_variable_err(w, lab, Xa.cpu().numpy().astype(np.float64).T, Xa_ref.T)
        eXb = per_variable_err(w, lab, Xb.cpu().numpy().astype(np.float64).T, Xb_ref.T)
        esq = float(np.max(np.abs(sq - sq_ref) / sq_ref))
        tol = 1e-9 if precision == 0 else 1e-4
        print(f"\ncycling {name} inflation={inflation} precision={precision}: RMSE {O.rmse_eq18(sq):.6e} "
              f"(oracle {O.rmse_eq18(sq_ref):.6e}) sqerr {esq:.2e} Xa {eXa:.2e} Xb {eXb:.2e}")
        assert esq < tol and eXa < tol and eXb < tol, (esq, eXa, eXb)
    finally:
        h.close()


def test_filter_run_graph_equals_eager(torch_cuda):
    """Cycles 1.. replay a captured graph; the same calls made one by one give
    the same bits."""
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    M, shift = 4, 2
    ci = make_cycle_inputs(w, M, shift, np.float32)
    dt = torch.float32
    out = []
    for graph in (True, False):
        h = _handle(torch, B, w, 1, ci.obs_idx)
        try:
            Xb, ys, Zs, R, xr = _inputs_on_device(torch, ci, dt)
            T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=dt)
            D = torch.empty(w.n, device="cuda", dtype=dt)
            Xa = torch.empty_like(Xb)
            sq = torch.zeros(M, dtype=torch.float64, device="cuda")
            if graph:
                h.filter_run(Xb, ys, Zs, R, xr, T, D, Xa, M, shift, sq)
            else:
                for k in range(M):
                    h.estimate(Xb, T, D)
                    h.assemble(Xb, T, D, R)
                    h.analyze(Xb, ys[k], R, Zs[k], Xa)
                    h.ensemble_sqerr(Xa, xr[k], sq[k:k + 1])
                    h.forecast_shift(Xa, Xb, w.N, shift)
            h.check()
            torch.cuda.synchronize()
            out.append((Xa.cpu().numpy(), Xb.cpu().numpy(), sq.cpu().numpy()))
        finally:
            h.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
