"""The dual form on the GPU (enkfmc_analyze_dual, Eq. 12-13) against the oracle.

The reference is the oracle's sub-domain analysis in the dual form (Eq.
12-13), pinned to its primal form by the Woodbury identity in
test_oracle_dual.py, on the same seeded inputs, at the tolerances of the
primal path (FP64 1e-9, FP32 1e-5, max |x - x_ref| / max |x_ref| per
variable).  (Against the oracle's primal form, FP64 would carry that form's
own rounding, amplified by the condition number of A: 1.9e-9 between the two
oracle forms on the ridge case.)  Cases: ragged tiles, the
longitude seam, the poles, 2-D and 3-D variables, r = 1, 2, 3, ridge rows, the
ill-conditioned blocks, sparse and denser networks, whole-ring and nearly
whole-ring boxes, a non-periodic grid, no observations; the T63 shape on one
sampled sub-domain; the shared-memory limit."""
import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_inputs
from _harness import TOL, gpu_pipeline, np_dtype, per_variable_err, torch_dtype

pytestmark = pytest.mark.gpu


def dual_pipeline(w, inp, precision, handle=None):
    """estimate -> analyze_dual on cuda:0 through the C ABI."""
    import torch
    from paper_1606_00807_gb300 import binding as B
    dt = torch_dtype(precision)
    h = handle or B.Handle.from_workload(w, precision=precision,
                                         stream=torch.cuda.current_stream().cuda_stream)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    Xb, y, R, Z = dev(inp.Xb), dev(inp.y), dev(inp.R), dev(inp.Z)
    T = torch.empty((w.n, h.info.pmax), device="cuda", dtype=dt)
    D = torch.empty(w.n, device="cuda", dtype=dt)
    Xa = torch.full_like(Xb, float("nan"))
    h.estimate(Xb, T, D)
    h.analyze_dual(Xb, T, D, y, R, Z, Xa)
    h.check()
    torch.cuda.synchronize()
    return dict(Xa=Xa.cpu().numpy().astype(np.float64), handle=h)


def oracle_xa(w, inp, only=None, form="dual"):
    f = lambda a: np.asarray(a, dtype=np.float64)
    return O.assimilate(w, f(inp.Xb), f(inp.y), f(inp.R), f(inp.Z), inp.obs_idx, only=only,
                        form=form)


def check(w, inp, got, ref, precision, labels=None):
    labels = np.arange(w.n) if labels is None else labels
    err = per_variable_err(w, labels, got[:, labels].T, ref[:, labels].T)
    dX, dXr = got[:, labels] - inp.Xb[:, labels], ref[:, labels] - inp.Xb[:, labels]
    err_dx = per_variable_err(w, labels, dX.T, dXr.T)
    assert np.abs(dXr).max() > 0
    assert err < TOL[precision], err
    # the increment on its own scale (a few times the analysis bound)
    assert err_dx < 10 * TOL[precision], err_dx
    return err, err_dx


CASES = [
    ("small_40x30x2x2+1_n48_r2", 0.1),      # ragged tiles, seam, poles, 2-D and 3-D
    ("small_48x26x3x1+1_n80_r2", 0.05),     # T63 statistics, sparse network
    ("small_40x30x0+2_n64_r3", 0.1),        # r = 3, one level
    ("small_28x20x3x1_n32_r1", 0.3),        # r = 1
    ("small_36x24x2x1_n24_r3_ridge", 0.1),  # ridge rows
    ("small_40x30x2x2+1_n24_r2_ill", 0.05), # blocks of A near kappa 1e11
    ("tiny_32x16_n20_r2", None),            # every second component observed
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,frac", CASES)
def test_dual_matches_oracle(name, frac, precision):
    w = WORKLOADS[name] if frac is None else WORKLOADS[name].with_(obs_frac=frac)
    inp = make_inputs(w, np_dtype(precision))
    out = dual_pipeline(w, inp, precision)
    check(w, inp, out["Xa"], oracle_xa(w, inp), precision)
    out["handle"].close()


@pytest.mark.parametrize("kw", [
    dict(nlon=16, sub_lon=16),          # whole-ring boxes starting past the seam
    dict(nlon=16, sub_lon=11),          # a box of 15 of the 16 longitudes
    dict(lon_periodic=False),           # no seam
])
def test_dual_box_shapes(kw):
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"].with_(obs_frac=0.15, **kw)
    for precision in (0, 1):
        inp = make_inputs(w, np_dtype(precision))
        out = dual_pipeline(w, inp, precision)
        check(w, inp, out["Xa"], oracle_xa(w, inp), precision)
        out["handle"].close()


def test_dual_equals_primal_on_gpu_and_is_reproducible():
    w = WORKLOADS["small_40x30x2x2+1_n48_r2"].with_(obs_frac=0.1)
    inp = make_inputs(w, np.float64)
    a = dual_pipeline(w, inp, 0)
    b = dual_pipeline(w, inp, 0, handle=a["handle"])
    assert np.array_equal(a["Xa"], b["Xa"])            # no atomics: same bits
    p = gpu_pipeline(w, inp, 0, handle=a["handle"])     # primal on the same handle
    assert per_variable_err(w, np.arange(w.n), a["Xa"].T, p["Xa"].T) < 1e-9
    prof = a["handle"].profile_read(kernels=True)
    for kind in ("dual_z", "dual_obs", "dual_apply"):
        assert prof[kind][1] > 0, kind
    work = a["handle"].work_per_launch()
    assert all(work[k][0] > 0 for k in ("dual_z", "dual_obs", "dual_apply"))
    a["handle"].close()


def test_dual_without_observations_is_identity():
    import torch
    w = WORKLOADS["small_28x20x3x1_n32_r1"]
    inp = make_inputs(w, np.float32)
    empty = inp.obs_idx[:0]
    from paper_1606_00807_gb300 import binding as B
    h = B.Handle.from_workload(w, precision=B.FP32)
    h.set_observations(empty)
    Xb = torch.from_numpy(inp.Xb).cuda()
    T = torch.empty((w.n, h.info.pmax), device="cuda")
    D = torch.empty(w.n, device="cuda")
    Xa = torch.full_like(Xb, float("nan"))
    h.estimate(Xb, T, D)
    h.analyze_dual(Xb, T, D, None, None, None, Xa)
    h.check()
    assert torch.equal(Xa, Xb)
    h.close()


def test_dual_limits_and_state():
    """A block whose observation system exceeds shared memory: EINVAL with nothing
    queued and nothing changed (an assembly stays valid); after the dual form,
    enkfmc_analyze needs a new enkfmc_assemble."""
    import torch
    from paper_1606_00807_gb300 import binding as B
    w = WORKLOADS["small_48x26x3x1+1_n80_r2"].with_(obs_frac=0.9)   # ~690 per block
    inp = make_inputs(w, np.float32)
    h = B.Handle.from_workload(w, precision=B.FP32)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Xb, y, R, Z = dev(inp.Xb), dev(inp.y), dev(inp.R), dev(inp.Z)
    T = torch.empty((w.n, h.info.pmax), device="cuda")
    D = torch.empty(w.n, device="cuda")
    Xa = torch.empty_like(Xb)
    h.estimate(Xb, T, D)
    h.assemble(Xb, T, D, R)
    with pytest.raises(B.EnkfmcError) as e:
        h.analyze_dual(Xb, T, D, y, R, Z, Xa)
    assert e.value.code == 1
    assert h.get_status()[0] == 0
    # the primal form still runs on the same handle, on the same assembly;
    # after a dual analysis it needs a new assembly
    h.analyze(Xb, y, R, Z, Xa)
    h.check()
    w2 = w.with_(obs_frac=0.05)
    inp2 = make_inputs(w2, np.float32)
    out = dual_pipeline(w2, inp2, 1, handle=h)
    with pytest.raises(B.EnkfmcError) as e:
        h.analyze(Xb, y, R, Z, Xa)
    assert e.value.code == 9
    check(w2, inp2, out["Xa"], oracle_xa(w2, inp2), 1)
    h.close()


def test_dual_t63_sampled_subdomain():
    """The T63 shape (192 x 96 x 29, N = 80, r = 2) with 4% of the components
    observed, in FP32: sub-domain 0 (the seam and the pole) against the oracle,
    and every component against the GPU primal form.  (The oracle's primal form
    here: its dense dual form would factor a 6,496-row sub-domain densely.)"""
    w = WORKLOADS["t63_192x96x29_n80_r2"].with_(obs_frac=0.04)
    inp = make_inputs(w, np.float32)
    out = dual_pipeline(w, inp, 1)
    ref = oracle_xa(w, inp, only=[0], form="primal")
    g = O.Grid.from_workload(w)
    sd0 = O.subdomains(g, w.sub_lon, w.sub_lat)[0]
    check(w, inp, out["Xa"], ref, 1, labels=sd0.interior)
    p = gpu_pipeline(w, inp, 1, handle=out["handle"])
    assert per_variable_err(w, np.arange(w.n), out["Xa"].T, p["Xa"].T) < 2 * TOL[1]
    out["handle"].close()
