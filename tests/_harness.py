"""Helpers shared by the GPU parity tests: run the library through its C ABI and
line its outputs up with the oracle's."""
from __future__ import annotations

import numpy as np

import oracle as O
from synthetic import Inputs, Workload

# Tolerances (max |x - x_ref| / max |x_ref| per variable, against the FP64 oracle).
# FP64 path: every step in double precision; rounding differences stay near
# 1e-13 relative for these condition numbers, 1e-9 leaves ample room.
# FP32 path: the target stated for single-precision paths, 1e-5.
TOL = {0: 1e-9, 1: 1e-5}


def torch_dtype(precision):
    import torch
    return torch.float64 if precision == 0 else torch.float32


def np_dtype(precision):
    return np.float64 if precision == 0 else np.float32


def gpu_pipeline(w: Workload, inp: Inputs, precision: int, handle=None, flags=0, tuning=None):
    """estimate -> assemble -> analyze on cuda:0 through the C ABI; returns numpy
    outputs.  tuning: {knob: value} for enkfmc_set_tuning."""
    import torch
    from paper_1606_00807_gb300 import binding as B
    dt = torch_dtype(precision)
    stream = torch.cuda.current_stream().cuda_stream
    h = handle or B.Handle.from_workload(w, precision=precision, stream=stream, flags=flags)
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
    h.check()
    torch.cuda.synchronize()
    return dict(T=T.cpu().numpy().astype(np.float64), D=D.cpu().numpy().astype(np.float64),
                Xa=Xa.cpu().numpy().astype(np.float64), handle=h)


def slot_neighbours(w: Workload, dk, dy, dx, rows: np.ndarray):
    """Label of the neighbour in every stencil slot of the given rows (ring
    longitude), or -1 where the slot leaves the grid."""
    g = O.Grid.from_workload(w)
    out = np.full((len(rows), len(dk)), -1, dtype=np.int64)
    for a, j in enumerate(rows):
        v, k, y, x = g.coords(int(j))
        for s in range(len(dk)):
            kk, yy, xx = k + dk[s], y + dy[s], x + dx[s]
            if kk < 0 or kk >= g.levels[v] or yy < 0 or yy >= g.nlat:
                continue
            if w.lon_periodic:
                xx %= g.nlon
            elif not 0 <= xx < g.nlon:
                continue
            out[a, s] = g.label(v, kk, yy, xx)
    return out


def max_block_condition(w: Workload, inp: Inputs) -> float:
    """Largest 2-norm condition number over the (sub-domain, variable) blocks of
    A = T^T D^-1 T + H^T R^-1 H, from the oracle in FP64."""
    from synthetic import variable_of
    g = O.Grid.from_workload(w)
    sds = O.subdomains(g, w.sub_lon, w.sub_lat)
    Xb = inp.Xb.T.astype(np.float64)
    U = O.anomalies(Xb)
    Ys = O.perturbed_observations(inp.y, inp.R, inp.Z.T)
    worst = 0.0
    for sd in sds:
        A, _, _, _, _ = O.local_system(g, sd, U, Xb, Ys, inp.R, inp.obs_idx, w.ridge_c)
        Ad = A.toarray()
        var = variable_of(w, sd.ext)
        for v in np.unique(var):
            sel = np.where(var == v)[0]
            ev = np.linalg.eigvalsh(Ad[np.ix_(sel, sel)])
            worst = max(worst, ev[-1] / ev[0])
    return worst


def per_variable_err(w: Workload, labels: np.ndarray, got: np.ndarray, ref: np.ndarray):
    """max over variables of max|got - ref| / max|ref|, rows grouped by variable."""
    from synthetic import variable_of
    var = variable_of(w, np.asarray(labels, dtype=np.int64))
    worst = 0.0
    for v in np.unique(var):
        sel = var == v
        worst = max(worst, O.rel_err(got[sel], ref[sel]))
    return worst


def elementwise_rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max_i |got_i - ref_i| / |ref_i| (ref_i != 0): every entry on its own scale, so a
    small D_j, whose inverse enters A, is held to the same relative bound as a large one."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if not ref.size:
        return 0.0
    assert np.all(ref != 0)
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def compare_T_rows(w: Workload, h, T_gpu: np.ndarray, D_gpu: np.ndarray, rows, ref_rows):
    """Errors against the oracle's (j, P, beta, D) rows: T per variable, D per variable
    and D element by element; also checks that every nonzero GPU coefficient sits on a
    predecessor.  Returns (eT, eD, eD_elem)."""
    dk, dy, dx = h.slot_offsets()
    rows = np.asarray(rows)
    nb = slot_neighbours(w, dk, dy, dx, rows)
    got = np.zeros((len(rows), len(dk)))
    ref = np.zeros((len(rows), len(dk)))
    dref = np.zeros(len(rows))
    for a, (j, P, beta, d) in enumerate(ref_rows):
        assert int(rows[a]) == j
        coef = {q: -b for q, b in zip(P, beta)}
        for s in range(len(dk)):
            q = int(nb[a, s])
            got[a, s] = T_gpu[j, s]
            ref[a, s] = coef.get(q, 0.0)
            if q not in coef:
                assert T_gpu[j, s] == 0.0, (j, s)
        dref[a] = d
    return (per_variable_err(w, rows, got, ref),
            per_variable_err(w, rows, D_gpu[rows], dref),
            elementwise_rel_err(D_gpu[rows], dref))
