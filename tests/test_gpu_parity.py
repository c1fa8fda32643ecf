"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-by-element comparisons on seeded inputs: the sparsity pattern of T
bit for bit, every T row and D entry, and the analysis ensemble, in FP64 and
FP32, on grids that span several tiles with ragged edges, the longitude seam
and the poles; at the T63 shape on sampled rows and sub-domains.
"""
import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_inputs

from _harness import (TOL, compare_T_rows, gpu_pipeline, max_block_condition, np_dtype,
                      per_variable_err)

pytestmark = pytest.mark.gpu

# both precisions at the fixed tolerances: sub-domain systems with kappa <= 6e3,
# and the N = 16, r = 1 case (p > N / 2 on most rows: regressions in double
# precision inside the single-precision path; kappa 1e7, four refinement steps)
SMALL = ["small_48x26x3x1+1_n80_r2", "small_40x30x2x2+1_n48_r2", "tiny_32x16_n20_r2",
         "small_28x20x3x1_n32_r1", "small_28x20x3x1_n16_r1"]
# p >= N - 1 on most rows (ridge): kappa 7e6 and 1.5e11
ILL = ["small_36x24x2x1_n24_r3_ridge", "small_40x30x2x2+1_n24_r2_ill"]
EPS64 = 2.0 ** -52


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00807_gb300 import binding
    binding.load()


@pytest.mark.parametrize("name", SMALL + ILL + ["nonperiodic"])
def test_T_pattern_bit_exact(name):
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS[SMALL[1]].with_(lon_periodic=False) if name == "nonperiodic" else WORKLOADS[name]
    h = B.Handle.from_workload(w, precision=B.FP64)
    rowptr, col = h.export_T_pattern()
    ref_ptr, ref_col = O.t_pattern_csr(O.Grid.from_workload(w))
    assert np.array_equal(rowptr, ref_ptr)
    assert np.array_equal(col, ref_col)
    h.close()


def _parity(name, precision, tol_x=None, flags=0, tuning=None):
    w = WORKLOADS[name]
    inp = make_inputs(w, np_dtype(precision))
    out = gpu_pipeline(w, inp, precision, flags=flags, tuning=tuning)
    tol = TOL[precision]
    tol_x = tol if tol_x is None else tol_x
    # step (a): every row of T and D against the oracle
    U = O.anomalies(inp.Xb.T)
    g = O.Grid.from_workload(w)
    rows = np.arange(g.n)
    ref = O.estimate_rows(g, U, rows, w.ridge_c)
    eT, eD, eDe = compare_T_rows(w, out["handle"], out["T"], out["D"], rows, ref)
    # steps (b)-(c): the analysis ensemble and its increment
    Xa_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    Xb = inp.Xb.astype(np.float64)
    lab = np.arange(w.n)
    eX = per_variable_err(w, lab, out["Xa"].T, Xa_ref.T)
    edX = per_variable_err(w, lab, (out["Xa"] - Xb).T, (Xa_ref - Xb).T)
    print(f"\nparity {name} precision={precision} flags={flags}: T {eT:.2e} D {eD:.2e} "
          f"D(elementwise) {eDe:.2e} Xa {eX:.2e} dX {edX:.2e} "
          f"fp64 blocks {out['handle'].fp64_blocks()}")
    assert eT < tol, eT
    assert eD < tol, eD
    assert eDe < tol, eDe
    assert eX < tol_x, eX
    assert edX < tol_x, edX
    nfb = out["handle"].fp64_blocks()
    out["handle"].close()
    return nfb


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", SMALL)
def test_estimate_and_analysis_parity(name, precision):
    _parity(name, precision)


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("name", ["small_48x26x3x1+1_n80_r2", "small_48x26x3x1+1_n120_r2",
                                  "small_40x30x0+2_n64_r3"])
def test_register_and_tiled_regressions_parity(name, kernel):
    """Single-precision regressions a row per warp (1, as the default), through
    the register kernel (2; 37-39 slots with the seam at N = 80 and N = 120, 27
    slots for r = 3 on one level) and two rows per warp (3), chosen by
    ENKFMC_TUNE_REGRESS_KERNEL, each element by element against the oracle at the
    FP32 tolerance."""
    from paper_1606_00807_gb300 import binding as B
    _parity(name, 1, tuning={B.TUNE_REGRESS_KERNEL: kernel})


def test_plain_fp32_form_parity():
    """ENKFMC_FLAG_PLAIN_FP32 with no refinement (the plain single-precision form)
    on the T63 statistics, where no row has 2p > N and no block needs double
    precision: element by element against the oracle at the FP32 tolerance."""
    from paper_1606_00807_gb300 import binding as B
    assert _parity("small_48x26x3x1+1_n80_r2", 1,
                   flags=B.FLAG_PLAIN_FP32 | B.FLAG_NO_SOLVE_REFINEMENT) == 0


def test_plain_fp32_form_has_no_double_precision_rows():
    """N = 16, r = 1 (p > N / 2 on most rows): the default regresses those rows in
    double precision; the plain form regresses every row in single precision."""
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_28x20x3x1_n16_r1"]
    for flags, want in ((0, 1), (B.FLAG_PLAIN_FP32, 0)):
        h = B.Handle.from_workload(w, precision=B.FP32, flags=flags)
        try:
            assert h.info.fp64_rows == want, flags
        finally:
            h.close()


def test_plain_fp32_solve_without_refinement():
    """The single-precision solve without its refinement step (the plain FP32 form)
    on the T63 statistics, where the sub-domain blocks are well conditioned."""
    _parity("small_48x26x3x1+1_n80_r2", 1, flags=1)


@pytest.mark.parametrize("flags", [2, 3])
def test_cuda_core_solve_parity(flags):
    """Single precision with the band Cholesky and solves on the CUDA cores only
    (ENKFMC_FLAG_SIMT_BAND), with (2) and without (3) the refinement step."""
    _parity("small_48x26x3x1+1_n80_r2", 1, flags=flags)


def test_tensor_core_and_cuda_core_solves_agree():
    """The TF32-split tensor-core factorisation and solves and the FP32 CUDA-core
    ones, both followed by the refinement step, give the same analysis to the FP32
    tolerance."""
    w = WORKLOADS["small_48x26x3x1+1_n80_r2"]
    inp = make_inputs(w, np.float32)
    a = gpu_pipeline(w, inp, 1)
    b = gpu_pipeline(w, inp, 1, flags=2)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["D"], b["D"])
    lab = np.arange(w.n)
    Xb = inp.Xb.astype(np.float64)
    err = per_variable_err(w, lab, (a["Xa"] - Xb).T, (b["Xa"] - Xb).T)
    assert err <= TOL[1], err


@pytest.mark.parametrize("name", ILL)
def test_ill_conditioned_fp64_parity(name):
    """T and D at the FP64 tolerance; the analysis within a bound derived from the
    conditioning: both solvers are backward stable, so their forward errors are
    O(kappa * eps) and the bound is 1e-9 + 50 kappa eps."""
    w = WORKLOADS[name]
    kappa = max_block_condition(w, make_inputs(w, np.float64))
    assert kappa > 1e6
    _parity(name, 0, tol_x=1e-9 + 50.0 * kappa * EPS64)


def test_ridge_fp32_parity():
    """The ridge case (p >= N - 1 on most rows, block condition numbers near 7e6) in
    single precision at the fixed FP32 tolerance: its regressions run in double
    precision (2p > N) and its sub-domain solves take four refinement steps."""
    _parity("small_36x24x2x1_n24_r3_ridge", 1)


def test_ill_fp32_parity_with_double_precision_blocks():
    """N = 24, r = 2 on the 40 x 30 grid: block condition numbers up to 1.5e11, beyond
    what a single-precision factorisation holds (some pivots turn non-positive).  The
    regressions run in double precision (2p > N); the blocks whose single-precision
    factorisation fails are assembled again and factored and solved in double
    precision; the analysis then matches the oracle at the FP32 tolerance (the
    single-precision storage of T and D alone moves dX by about 4e-6 here)."""
    nfb = _parity("small_40x30x2x2+1_n24_r2_ill", 1)
    assert nfb > 0, "no block took the double-precision factorisation"


def test_indefinite_A_reports_enotspd_without_trap():
    """Negated observation variances make A indefinite: the single-precision and the
    double-precision factorisations both meet a non-positive pivot, and the library
    reports ENOTSPD with the failing block (no trap); the context stays usable."""
    import torch
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w, np.float32)
    h = B.Handle.from_workload(w, precision=B.FP32, stream=torch.cuda.current_stream().cuda_stream)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Xb, R = dev(inp.Xb), dev(-inp.R)
    T = torch.empty((w.n, h.info.pmax), device="cuda")
    D = torch.empty(w.n, device="cuda")
    h.estimate(Xb, T, D)
    h.assemble(Xb, T, D, R)
    code, info = h.get_status()
    assert code == 3 and 0 <= info < h.info.nblock, (code, info)
    h.assemble(Xb, T, D, dev(inp.R))
    assert h.get_status()[0] == 0 and h.fp64_blocks() == 0
    h.close()


@pytest.mark.parametrize("name", ["t63_192x96x29_n80_r2", "t63_192x96x29_n40_r2"])
def test_full_t63_sampled_fp32(name):
    """T63 shape, FP32, in the launch configuration the benchmark times: sampled T
    rows and D entries, and three sampled sub-domains of the analysis.  N = 80 is
    the headline workload; N = 40 (p = 37 of 39 degrees of freedom on interior
    rows) is the forward + adjoint workload, whose regressions run in double
    precision and whose solves take four refinement steps."""
    w = WORKLOADS[name]
    inp = make_inputs(w, np.float32)
    out = gpu_pipeline(w, inp, 1)
    g = O.Grid.from_workload(w)
    U = O.anomalies(inp.Xb.T)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([
        rng.choice(g.n, 300, replace=False),
        [0, w.nlon - 1, w.nlon, g.n - 1, g.offsets[4], g.offsets[4] + w.nlon - 1,
         g.offsets[1] - 1, g.label(2, 3, 47, 191), g.label(3, 6, 95, 0)]]))
    ref = O.estimate_rows(g, U, rows, w.ridge_c)
    eT, eD, eDe = compare_T_rows(w, out["handle"], out["T"], out["D"], rows, ref)
    print(f"\n{name} sampled rows: T {eT:.2e} D {eD:.2e} D(elementwise) {eDe:.2e}; "
          f"{out['handle'].fp64_blocks()} blocks factored in double precision")
    assert eT < TOL[1], eT
    assert eD < TOL[1], eD
    assert eDe < TOL[1], eDe
    # sub-domains: pole + seam corner, an interior tile, the last tile
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    pick = [0, 16 * 3 + 7, len(sds) - 1]
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    Xa_ref = O.analysis(g, sds, inp.Xb.T.astype(np.float64), Ys, inp.R, inp.obs_idx, w.ridge_c,
                        only=pick)
    for i in pick:
        lab = sds[i].interior
        got = out["Xa"][:, lab].T
        eX = per_variable_err(w, lab, got, Xa_ref[lab])
        edX = per_variable_err(w, lab, got - inp.Xb[:, lab].T, Xa_ref[lab] - inp.Xb[:, lab].T)
        print(f"{name} sub-domain {i}: Xa {eX:.2e} dX {edX:.2e}")
        assert eX < TOL[1], (i, eX)
        assert edX < TOL[1], (i, edX)
    out["handle"].close()


def test_no_observations_leaves_ensemble_unchanged():
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"].with_(obs="none")
    inp = make_inputs(w, np.float64)
    out = gpu_pipeline(w, inp, 0)
    assert np.array_equal(out["Xa"], inp.Xb)
    out["handle"].close()


def test_deterministic_and_host_cycle_matches():
    import torch
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_48x26x3x1+1_n80_r2"]
    inp = make_inputs(w, np.float32)
    a = gpu_pipeline(w, inp, 1)
    b = gpu_pipeline(w, inp, 1, handle=a["handle"])
    assert np.array_equal(a["Xa"], b["Xa"]) and np.array_equal(a["T"], b["T"])
    Xa = np.empty_like(inp.Xb)
    a["handle"].cycle_host(inp.Xb, inp.y, inp.R, inp.Z, Xa)
    assert np.array_equal(Xa.astype(np.float64), a["Xa"])
    # page-locked buffers: y, R and Z arrive on the copy stream during the
    # estimate; twice in a row, the second call's copies behind the first's work
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hXb, hy, hR, hZ = pin(inp.Xb), pin(inp.y), pin(inp.R), pin(inp.Z)
    for _ in range(2):
        hXa = torch.full_like(hXb, float("nan")).pin_memory()
        a["handle"].cycle_host(hXb, hy, hR, hZ, hXa)
        assert np.array_equal(hXa.numpy().astype(np.float64), a["Xa"])
    a["handle"].close()


def test_invalid_arguments_rejected_synchronously():
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["tiny_32x16_n20_r2"]
    with pytest.raises(B.EnkfmcError) as e:
        B.Handle.from_workload(w.with_(nlon=4))            # nlon < 2r + 1
    assert e.value.code == 1
    with pytest.raises(B.EnkfmcError):
        B.Handle.from_workload(w.with_(N=1))
    h = B.Handle.from_workload(w, precision=B.FP64)
    for bad in ([3, 2], [0, 0], [-1], [w.n]):
        with pytest.raises(B.EnkfmcError) as e:
            h.set_observations(np.array(bad, np.int32))
        assert e.value.code == 1
    import torch
    X = torch.zeros((w.N, w.n), device="cuda", dtype=torch.float64)
    with pytest.raises(B.EnkfmcError) as e:          # assemble before set_observations
        h.assemble(X, X, X, X)
    assert e.value.code == 9
    h.close()


def test_nonfinite_input_reports_status_not_trap():
    import torch
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w, np.float64)
    inp.Xb[3, 100] = np.nan
    h = B.Handle.from_workload(w, precision=B.FP64, stream=torch.cuda.current_stream().cuda_stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    Xb = dev(inp.Xb)
    T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=torch.float64)
    D = torch.empty(w.n, device="cuda", dtype=torch.float64)
    h.estimate(Xb, T, D)
    code, info = h.get_status()
    assert code in (4, 5)
    # the context stays usable: a clean run afterwards succeeds
    h.estimate(dev(make_inputs(w, np.float64).Xb), T, D)
    assert h.get_status()[0] == 0
    h.close()


def test_band_too_wide_for_the_band_kernels_is_refused():
    """A 24 x 24 tile with r = 3 on three levels gives a band about 990 wide,
    beyond the double-precision band kernels' shared memory (the pool of an FP32
    problem uses them): enkfmc_create refuses it with EINVAL instead of failing
    at launch; the plain FP32 form (no double-precision blocks) is accepted."""
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["study_96x48x3x2+1_n60"].with_(r=3, sub_lon=24, sub_lat=24)
    with pytest.raises(B.EnkfmcError) as ei:
        B.Handle.from_workload(w, precision=B.FP32)
    assert "EINVAL" in str(ei.value)
    h = B.Handle.from_workload(w, precision=B.FP32, flags=B.FLAG_PLAIN_FP32)
    assert h.info.hb_max > 900
    h.close()
