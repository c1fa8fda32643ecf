"""The allocation-free estimate, enkfmc_estimate_noalloc, through the C ABI.

Some callers cannot let the library allocate device memory: a service that
reserves its whole GPU memory budget up front, a host application whose own
allocator owns the device, or a latency-critical loop that cannot afford the
device-wide synchronisation cudaMalloc/cudaFree may cause.  For them the
library offers one entry point whose only scratch is a fixed 16 MiB device
array inside the library.

Checked here, each time with two calls in a row on different ensembles (the
second call must not see anything the first left in the shared array):
  * T and D equal, bit for bit, what the handle-based enkfmc_estimate writes
    for the same problem and ensemble (the same kernels on the same inputs);
  * T and D match the FP64 oracle at the tolerances of the parity tests;
  * single precision, double precision, and a single-precision problem whose
    rows with 2p > N are regressed in double precision (more scratch);
  * a problem just under the 16 MiB limit runs; one just over it is refused
    with EINVAL and leaves the outputs untouched.

The file name sorts last, so a run that stops at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, Workload, make_inputs

from _harness import TOL, compare_T_rows

pytestmark = pytest.mark.gpu

LIMIT = 16 << 20

# One 3-D variable on 3 levels, r = 2, N = 80 (no row with 2p > N): the single-
# precision scratch is round256(4 n 80) + round256(4 n 122) bytes.  96 x 72 x 3
# components need 16,754,688 bytes (22.5 KB below the limit); 96 x 73 x 3 need
# 16,987,392 (over it).
NEAR = Workload(name="noalloc_96x72x3_n80_r2", nlon=96, nlat=72, nlev=3, nvar_3d=1, nvar_2d=0,
                r=2, N=80, sub_lon=12, sub_lat=12, sigma2=(4.0,), corr_len=3.0, seed=9100)
OVER = NEAR.with_(name="noalloc_96x73x3_n80_r2", nlat=73)


def _need_fp32(w):
    r256 = lambda b: (b + 255) // 256 * 256
    return r256(4 * w.n * 80) + r256(4 * w.n * 122)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _both(torch, B, w, precision, inp):
    """(noalloc T, D), (handle T, D) as numpy, for one ensemble."""
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
    out = (T.cpu().numpy(), D.cpu().numpy(), T_ref.cpu().numpy(), D_ref.cpu().numpy(), h)
    return out


def _check_pair(torch, B, w, precision, rows=None):
    """Two calls in a row (seeds w.seed and w.seed + 1): bitwise against the handle,
    and against the oracle on `rows` (all rows when None)."""
    npdt = np.float64 if precision == B.FP64 else np.float32
    for wk in (w, w.with_(seed=w.seed + 1)):
        inp = make_inputs(wk, npdt)
        T, D, T_ref, D_ref, h = _both(torch, B, wk, precision, inp)
        assert np.all(np.isfinite(D))
        assert np.array_equal(T, T_ref), "T differs from enkfmc_estimate"
        assert np.array_equal(D, D_ref), "D differs from enkfmc_estimate"
        g = O.Grid.from_workload(wk)
        sel = np.arange(g.n) if rows is None else rows
        ref = O.estimate_rows(g, O.anomalies(inp.Xb.T), sel, wk.ridge_c)
        eT, eD, eDe = compare_T_rows(wk, h, T.astype(np.float64), D.astype(np.float64), sel, ref)
        tol = TOL[precision]
        assert max(eT, eD, eDe) < tol, (wk.name, precision, eT, eD, eDe)
        h.close()


def test_noalloc_matches_handle_and_oracle_two_calls(torch_cuda):
    from paper_1606_00807_gb300 import binding as B
    _check_pair(torch_cuda, B, WORKLOADS["small_48x26x3x1+1_n80_r2"], B.FP32)
    _check_pair(torch_cuda, B, WORKLOADS["tiny_32x16_n20_r2"], B.FP64)
    # 2p > N on most rows: the double-precision rows and their FP64 scratch
    _check_pair(torch_cuda, B, WORKLOADS["small_28x20x3x1_n16_r1"], B.FP32)


def test_noalloc_just_under_the_limit_runs(torch_cuda):
    from paper_1606_00807_gb300 import binding as B
    assert _need_fp32(NEAR) <= LIMIT < _need_fp32(OVER)
    rows = np.random.default_rng(3).choice(NEAR.n, 300, replace=False)
    rows = np.unique(np.concatenate([rows, [0, NEAR.n - 1]]))
    _check_pair(torch_cuda, B, NEAR, B.FP32, rows=rows)


def test_noalloc_just_over_the_limit_is_refused(torch_cuda):
    from paper_1606_00807_gb300 import binding as B
    torch = torch_cuda
    lib = B.load()
    w = OVER
    prob = B.enkfmc_problem(w.nlon, w.nlat, w.nlev, w.nvar_3d, w.nvar_2d, 1, w.r, w.vert_reach,
                            w.N, w.sub_lon, w.sub_lat, B.FP32, w.ridge_c, 0)
    Xb = torch.zeros((w.N, w.n), device="cuda")
    T = torch.full((w.n, 39), 7.0, device="cuda")
    D = torch.full((w.n,), 7.0, device="cuda")
    assert lib.enkfmc_estimate_noalloc(ctypes.byref(prob), Xb.data_ptr(), T.data_ptr(),
                                       D.data_ptr(), None) == 1
    torch.cuda.synchronize()
    assert bool((T == 7.0).all()) and bool((D == 7.0).all())     # nothing was queued
    big = WORKLOADS["t63_192x96x29_n80_r2"]                        # far beyond the limit
    prob = B.enkfmc_problem(big.nlon, big.nlat, big.nlev, big.nvar_3d, big.nvar_2d, 1, big.r,
                            big.vert_reach, big.N, big.sub_lon, big.sub_lat, B.FP32, big.ridge_c, 0)
    assert lib.enkfmc_estimate_noalloc(ctypes.byref(prob), Xb.data_ptr(), T.data_ptr(),
                                       D.data_ptr(), None) == 1
