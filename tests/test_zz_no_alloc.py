"""The allocation-free estimate, enkfmc_estimate_noalloc, against enkfmc_estimate.

Some callers cannot let the library allocate device memory: a service that
reserves its whole GPU memory budget up front, a host application whose own
allocator owns the device, or a latency-critical loop that cannot afford the
device-wide synchronisation cudaMalloc/cudaFree may cause.  For them the
library offers one entry point whose only scratch is a fixed device array
inside the library.  This test calls it twice in a row through the C ABI, on
two different ensembles, and checks each result against the handle-based
enkfmc_estimate within the tolerances the parity tests use.  It also checks
that a problem too large for the fixed array is refused before any work runs.

The file name sorts last, so a run that stops at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _estimate_both(torch, B, w, precision, inp):
    dt = torch.float64 if precision == B.FP64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    h = B.Handle.from_workload(w, precision=precision, stream=stream)
    Xb = torch.from_numpy(np.ascontiguousarray(inp.Xb)).to("cuda", dt)
    T_ref = torch.empty((w.n, h.info.pmax), device="cuda", dtype=dt)
    D_ref = torch.empty(w.n, device="cuda", dtype=dt)
    h.estimate(Xb, T_ref, D_ref)
    h.check("enkfmc_estimate")
    T = torch.full_like(T_ref, float("nan"))
    D = torch.full_like(D_ref, float("nan"))
    rc = h.lib.enkfmc_estimate_noalloc(ctypes.byref(h.problem), Xb.data_ptr(), T.data_ptr(),
                                       D.data_ptr(), ctypes.c_void_p(stream))
    assert rc == 0, B.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    out = (T.cpu().numpy(), D.cpu().numpy(), T_ref.cpu().numpy(), D_ref.cpu().numpy())
    h.close()
    return out


def test_noalloc_estimate_matches_handle_estimate_two_calls(torch_cuda):
    from paper_1606_00807_gb300 import binding as B
    torch = torch_cuda
    base = WORKLOADS["small_48x26x3x1+1_n80_r2"]
    cases = [(base, B.FP32, 1e-5), (base.with_(seed=base.seed + 1), B.FP32, 1e-5)]
    for w, precision, tol in cases:            # two calls in a row on the shared array
        inp = make_inputs(w, np.float32 if precision == B.FP32 else np.float64)
        T, D, T_ref, D_ref = _estimate_both(torch, B, w, precision, inp)
        assert np.all(np.isfinite(D))
        assert O.rel_err(T, T_ref) <= tol
        assert O.rel_err(D, D_ref) <= tol
    w = WORKLOADS["tiny_32x16_n20_r2"]
    inp = make_inputs(w, np.float64)
    T, D, T_ref, D_ref = _estimate_both(torch, B, w, B.FP64, inp)
    assert O.rel_err(T, T_ref) <= 1e-9 and O.rel_err(D, D_ref) <= 1e-9


def test_noalloc_rejects_problem_beyond_scratch(torch_cuda):
    from paper_1606_00807_gb300 import binding as B
    lib = B.load()
    w = WORKLOADS["t63_192x96x29_n80_r2"]        # 534,528 x 80 floats: far beyond 16 MiB
    prob = B.enkfmc_problem(w.nlon, w.nlat, w.nlev, w.nvar_3d, w.nvar_2d, 1, w.r, w.vert_reach,
                            w.N, w.sub_lon, w.sub_lat, B.FP32, w.ridge_c)
    dummy = torch_cuda.empty(1, device="cuda")
    p = dummy.data_ptr()
    assert lib.enkfmc_estimate_noalloc(ctypes.byref(prob), p, p, p, None) == 1
