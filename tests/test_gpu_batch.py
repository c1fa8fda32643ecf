"""Batches of independent problems of uneven size in one CUDA graph
(enkfmc_batch_*), and the launch autotuner.

The instances are the first ones of the 256-instance set (grids from 24 x 12 to
96 x 48, 1-7 levels, 1-5 variables, N in [20, 120], r in {1, ..., 4}).  Checked:
a graph replay writes exactly what each handle writes when run on its own;
the per-problem status array is clean; sampled instances match the FP64 oracle
element by element at the FP32 tolerance (T, D per variable and element-wise,
X^a and dX per variable); the autotuner's choice does not change the results.
"""
import numpy as np
import pytest

import oracle as O
from synthetic import make_inputs
from synthetic.workloads import batch_instances

from _harness import TOL, compare_T_rows, per_variable_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _instance(torch, B, w, flags=0):
    inp = make_inputs(w, np.float32)
    h = B.Handle.from_workload(w, precision=B.FP32,
                               stream=torch.cuda.current_stream().cuda_stream, flags=flags)
    h.set_observations(inp.obs_idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bufs = dict(Xb=dev(inp.Xb), y=dev(inp.y), R=dev(inp.R), Z=dev(inp.Z),
                T=torch.empty((w.n, h.info.pmax), device="cuda"),
                D=torch.empty(w.n, device="cuda"))
    bufs["Xa"] = torch.empty_like(bufs["Xb"])
    return inp, h, bufs


def _eager(h, b):
    h.estimate(b["Xb"], b["T"], b["D"])
    h.assemble(b["Xb"], b["T"], b["D"], b["R"])
    h.analyze(b["Xb"], b["y"], b["R"], b["Z"], b["Xa"])


def test_batch_graph_equals_eager_and_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1606_00807_gb300 import binding as B
    ws = batch_instances()[:16]
    insts = [_instance(torch, B, w) for w in ws]
    try:
        _graph_equals_eager_and_oracle(torch, B, ws, insts)
    finally:
        for _, h, _ in insts:
            h.close()


def _graph_equals_eager_and_oracle(torch, B, ws, insts):
    eager = []
    for w, (inp, h, b) in zip(ws, insts):
        _eager(h, b)
        h.check(w.name)
        eager.append((b["Xa"].cpu().numpy().copy(), b["T"].cpu().numpy().copy(),
                      b["D"].cpu().numpy().copy()))
        b["Xa"].fill_(float("nan"))
    batch = B.Batch([h for _, h, _ in insts], nstreams=4,
                    stream=torch.cuda.current_stream().cuda_stream)
    for i, (inp, h, b) in enumerate(insts):
        batch.bind(i, b["Xb"], b["T"], b["D"], b["y"], b["R"], b["Z"], b["Xa"])
    batch.capture()
    for i, (_, _, b) in enumerate(insts):
        b["Xa"].fill_(float("nan"))
    for _ in range(2):
        batch.run()
    st, info = batch.status()
    assert not st.any(), (st, info)
    ns, of = batch.streams()
    assert ns == 4 and set(of.tolist()) <= set(range(4))
    for i, (w, (inp, h, b)) in enumerate(zip(ws, insts)):
        assert np.array_equal(b["Xa"].cpu().numpy(), eager[i][0]), w.name
        assert np.array_equal(b["T"].cpu().numpy(), eager[i][1]), w.name
    # the smallest four against the oracle, element by element
    small = sorted(range(len(ws)), key=lambda i: ws[i].n * ws[i].N)[:4]
    for i in small:
        w, (inp, h, b) = ws[i], insts[i]
        g = O.Grid.from_workload(w)
        rows = np.arange(g.n)
        ref = O.estimate_rows(g, O.anomalies(inp.Xb.T), rows, w.ridge_c)
        eT, eD, eDe = compare_T_rows(w, h, eager[i][1].astype(np.float64),
                                     eager[i][2].astype(np.float64), rows, ref)
        Xa_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
        Xa = b["Xa"].cpu().numpy().astype(np.float64)
        lab = np.arange(w.n)
        eX = per_variable_err(w, lab, Xa.T, Xa_ref.T)
        edX = per_variable_err(w, lab, (Xa - inp.Xb).T, (Xa_ref - inp.Xb).T)
        print(f"\nbatch instance {w.name}: T {eT:.2e} D {eD:.2e} D(elementwise) {eDe:.2e} "
              f"Xa {eX:.2e} dX {edX:.2e} fp64 blocks {h.fp64_blocks()}")
        assert max(eT, eD, eDe, eX, edX) < TOL[1], (w.name, eT, eD, eDe, eX, edX)
    batch.close()


def test_autotuner_choice_leaves_results_unchanged(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_1606_00807_gb300 import autotune, binding as B
    w = batch_instances()[2]
    inp, h, b = _instance(torch, B, w)
    try:
        _eager(h, b)
        h.check()
    finally:
        h.close()
    ref = b["Xa"].cpu().numpy().copy()
    cache = {}
    bufs = (b["Xb"], b["T"], b["D"], b["y"], b["R"], b["Z"], b["Xa"])
    choice = autotune.tune(w, inp.obs_idx, bufs, cache=cache)
    assert set(choice) >= {"flags", "regress_cap", "ms", "timings"}
    assert len(choice["timings"]) == len(autotune.BAND_PATHS) * len(autotune.REGRESS_CAPS)
    path = str(tmp_path / "tune.json")
    autotune.save_cache(cache, path)
    assert autotune.load_cache(path)[autotune.shape_key(w, B.FP32)]["flags"] == choice["flags"]
    h2 = B.Handle.from_workload(w, precision=B.FP32,
                                stream=torch.cuda.current_stream().cuda_stream,
                                flags=choice["flags"])
    try:
        h2.set_observations(inp.obs_idx)
        autotune.apply(h2, choice)
        _eager(h2, b)
        h2.check()
    finally:
        h2.close()
    got = b["Xa"].cpu().numpy()
    if choice["flags"] == 0:
        assert np.array_equal(got, ref)       # same kernels, another grid cap
    else:                                      # CUDA-core band path: same analysis to FP32
        assert per_variable_err(w, np.arange(w.n), (got - inp.Xb).T, (ref - inp.Xb).T) < TOL[1]
