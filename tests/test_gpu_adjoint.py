"""Reverse pass on the GPU (enkfmc_analyze_adjoint) against the FP64 oracle's
gradient (itself pinned by central differences), a GPU finite-difference check
in FP64, and the torch.autograd.Function path."""
import numpy as np
import pytest

import oracle as O
from oracle.adjoint import analysis_with_gradient, loss_mean_analysis
from synthetic import WORKLOADS, make_inputs

from _harness import np_dtype, torch_dtype

pytestmark = pytest.mark.gpu

# FP64: rounding order only.  FP32: the reverse solves are refined like the
# forward ones, but the recomputed Gram factors of the single-precision rows
# solve v = (G + lambda I)^-1 betabar in single precision without refinement
# (measured at most 5.5e-6 on the small cases).  At T63 with N = 40 the Gram
# matrices reach condition numbers near 1e8 and the reverse pass reads T, D,
# dX and Lambda stored in single precision: 1e-3 there (measured 5.2e-4).
TOL = {0: 1e-9, 1: 1e-4}
TOL_T63_N40 = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gpu_grad(torch, w, inp, precision, seed, tuning=None):
    from paper_1606_00807_gb300 import binding as B
    dt = torch_dtype(precision)
    h = B.Handle.from_workload(w, precision=precision,
                               stream=torch.cuda.current_stream().cuda_stream)
    for knob, value in (tuning or {}).items():
        h.set_tuning(knob, value)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    Xb, y, R, Z = dev(inp.Xb), dev(inp.y), dev(inp.R), dev(inp.Z)
    T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=dt)
    D = torch.empty(w.n, device="cuda", dtype=dt)
    Xa = torch.empty_like(Xb)
    h.estimate(Xb, T, D)
    h.assemble(Xb, T, D, R)
    h.analyze(Xb, y, R, Z, Xa)
    W = dev(seed)
    Xb_bar, y_bar, R_bar = torch.empty_like(Xb), torch.empty_like(y), torch.empty_like(R)
    h.analyze_adjoint(W, y_bar, R_bar, Xb_bar)
    h.check("adjoint")
    torch.cuda.synchronize()
    out = [a.cpu().numpy().astype(np.float64) for a in (Xa, Xb_bar, y_bar, R_bar)]
    h.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["tiny_32x16_n20_r2", "small_48x26x3x1+1_n80_r2",
                                  "small_40x30x2x2+1_n48_r2"])
def test_adjoint_matches_oracle(torch_cuda, name, precision):
    w = WORKLOADS[name]
    inp = make_inputs(w, np_dtype(precision))
    Xa_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    _, W = loss_mean_analysis(Xa_ref, inp.truth)   # dL/dXa of the mean-analysis loss
    W = W + 0.01 * np.random.default_rng(2).standard_normal(W.shape)  # and a generic part
    W = W.astype(np_dtype(precision))
    _, Xb_bar, y_bar, R_bar = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z,
                                                     inp.obs_idx, W)
    got = _gpu_grad(torch_cuda, w, inp, precision, W)
    errs = {k: O.rel_err(g, r) for k, g, r in (("Xb", got[1], Xb_bar), ("y", got[2], y_bar),
                                               ("R", got[3], R_bar))}
    print(f"\nadjoint {name} precision={precision}: " +
          " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < TOL[precision], (k, v)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_regression_kernels_match_oracle(torch_cuda, kernel):
    """FP32 reverse pass with the tiled (1) and the register-resident (2)
    regression adjoint (ENKFMC_TUNE_REGRESS_KERNEL) on the T63 statistics
    (37-39 slots), each against the oracle's gradient."""
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_48x26x3x1+1_n80_r2"]
    inp = make_inputs(w, np.float32)
    Xa_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    _, W = loss_mean_analysis(Xa_ref, inp.truth)
    W = (W + 0.01 * np.random.default_rng(3).standard_normal(W.shape)).astype(np.float32)
    _, Xb_bar, y_bar, R_bar = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z,
                                                     inp.obs_idx, W)
    got = _gpu_grad(torch_cuda, w, inp, 1, W, tuning={B.TUNE_REGRESS_KERNEL: kernel})
    errs = {k: O.rel_err(g, r) for k, g, r in (("Xb", got[1], Xb_bar), ("y", got[2], y_bar),
                                               ("R", got[3], R_bar))}
    print(f"\nadjoint kernel {kernel}: " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < TOL[1], (k, v)


def test_gpu_gradient_matches_gpu_finite_differences(torch_cuda):
    """FP64 on the GPU: central differences of L = 1/2 |mean(X^a) - x_ref|^2 computed
    by the GPU forward against the GPU reverse pass, in random directions."""
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w, np.float64)

    def loss(Xb, y, R):
        h = B.Handle.from_workload(w, precision=B.FP64,
                                   stream=torch.cuda.current_stream().cuda_stream)
        h.set_observations(inp.obs_idx)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
        X, yy, RR, Z = dev(Xb), dev(y), dev(R), dev(inp.Z)
        T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=torch.float64)
        D = torch.empty(w.n, device="cuda", dtype=torch.float64)
        Xa = torch.empty_like(X)
        h.estimate(X, T, D)
        h.assemble(X, T, D, RR)
        h.analyze(X, yy, RR, Z, Xa)
        h.check()
        L, Wb = loss_mean_analysis(Xa.cpu().numpy(), inp.truth)
        h.close()
        return L, Wb

    L0, W = loss(inp.Xb, inp.y, inp.R)
    _, gX, gy, gR = _gpu_grad(torch, w, inp, 0, W)
    rng = np.random.default_rng(9)
    for name, d, grad in (("Xb", rng.standard_normal(inp.Xb.shape), gX),
                          ("y", rng.standard_normal(inp.y.shape), gy),
                          ("R", rng.standard_normal(inp.R.shape) * inp.R, gR)):
        h = 1e-6
        args = [inp.Xb, inp.y, inp.R]
        k = {"Xb": 0, "y": 1, "R": 2}[name]
        ap = [a + h * d if i == k else a for i, a in enumerate(args)]
        am = [a - h * d if i == k else a for i, a in enumerate(args)]
        fd = (loss(*ap)[0] - loss(*am)[0]) / (2 * h)
        an = float(np.sum(grad * d))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-10 * L0, (name, fd, an)


def test_autograd_function(torch_cuda):
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    from paper_1606_00807_gb300.autograd import analysis
    w = WORKLOADS["small_48x26x3x1+1_n80_r2"]
    inp = make_inputs(w, np.float64)
    h = B.Handle.from_workload(w, precision=B.FP64)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    Xb = dev(inp.Xb).requires_grad_(True)
    y = dev(inp.y).requires_grad_(True)
    R = dev(inp.R).requires_grad_(True)
    Z = dev(inp.Z)
    x_ref = dev(inp.truth)
    Xa = analysis(Xb, y, R, Z, h)
    L = 0.5 * ((Xa.mean(0) - x_ref) ** 2).sum()
    L.backward()
    _, W = loss_mean_analysis(Xa.detach().cpu().numpy(), inp.truth)
    _, rX, ry, rR = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, W)
    assert O.rel_err(Xb.grad.cpu().numpy(), rX) < 1e-9
    assert O.rel_err(y.grad.cpu().numpy(), ry) < 1e-9
    assert O.rel_err(R.grad.cpu().numpy(), rR) < 1e-9
    h.close()


@pytest.mark.parametrize("name", ["t63_192x96x29_n40_r2"])
def test_adjoint_t63_one_subdomain_seed(torch_cuda, name):
    """T63 shape with N = 40 (the forward + adjoint workload), FP32: a seed dL/dX^a that
    vanishes outside one sub-domain's interior (a random field there), so the oracle's
    reference gradient needs that sub-domain only (the others contribute exactly
    zero); dL/dX^b, dL/dy and dL/d diag(R) against it over every component."""
    w = WORKLOADS[name]
    inp = make_inputs(w, np.float32)
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    k0 = 55
    W = np.zeros((w.N, w.n), np.float32)
    W[:, sds[k0].interior] = np.random.default_rng(4).standard_normal(
        (w.N, len(sds[k0].interior))).astype(np.float32)
    _, Xb_bar, y_bar, R_bar = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z,
                                                     inp.obs_idx, W, only=[k0])
    got = _gpu_grad(torch_cuda, w, inp, 1, W)
    errs = {k: O.rel_err(gv, r) for k, gv, r in (("Xb", got[1], Xb_bar), ("y", got[2], y_bar),
                                                 ("R", got[3], R_bar))}
    print(f"\nadjoint {name} one sub-domain seed: " +
          " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < TOL_T63_N40, (k, v)


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_is_reproducible_bit_for_bit(torch_cuda, precision):
    """Every sum of the reverse pass runs in a fixed order (no atomics): two runs of
    forward + adjoint on the same inputs give bit-identical gradients."""
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"]
    inp = make_inputs(w, np_dtype(precision))
    W = np.random.default_rng(3).standard_normal((w.N, w.n)).astype(np_dtype(precision))
    a = _gpu_grad(torch_cuda, w, inp, precision, W)
    b = _gpu_grad(torch_cuda, w, inp, precision, W)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
