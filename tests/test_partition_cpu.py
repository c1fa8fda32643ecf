"""The latitude-band partition of one analysis over two ranks, on CPU (gloo).

Each rank owns a band of sub-domain rows, receives the background rows its
local grid needs from its neighbours (one halo scatter), analyses the local
grid with the FP64 oracle standing in for the per-rank compute, and the owned
rows are gathered.  The reverse pass sends the gradient on rows a neighbour
owns back to it (halo reduce) and sums the observation gradients.  Checked
against the single-process oracle: the scattered background, X^a (primal and
dual form), and the gradients of L = 1/2 |mean(X^a) - x_ref|^2 with respect to
X^b, y and diag(R).
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORKLOAD = "small_40x30x2x2+1_n48_r2"


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from oracle.adjoint import analysis_with_gradient, loss_mean_analysis
        from paper_1606_00807_gb300 import partition as Pt
        from synthetic import WORKLOADS, make_inputs

        w = WORKLOADS[WORKLOAD]
        inp = make_inputs(w)
        bands = Pt.band_plan(w, world)
        b = bands[rank]
        # only the owned band of the background is this rank's own data
        X_own = Pt.grid_view(inp.Xb, w)[:, :, b.lat0:b.lat1].copy()
        X_loc = Pt.halo_scatter(dist, w, bands, rank, X_own)
        scatter_ok = np.array_equal(X_loc, Pt.grid_view(inp.Xb, w)[:, :, b.lo:b.hi])
        wl = Pt.local_workload(w, b)
        pos, lab = Pt.local_observations(w, b, inp.obs_idx)
        Xl = X_loc.reshape(w.N, -1)
        Xa_loc = O.assimilate(wl, Xl, inp.y[pos], inp.R[pos], inp.Z[:, pos], lab)
        Xa_band = Pt.grid_view(Xa_loc, wl)[:, :, b.lat0 - b.lo:b.lat1 - b.lo]
        Xa = Pt.gather_owned(dist, w, bands, rank, Xa_band)
        # the same partition with the dual form of the local analyses (Eq. 12-13)
        Xd_loc = O.assimilate(wl, Xl, inp.y[pos], inp.R[pos], inp.Z[:, pos], lab, form="dual")
        Xd = Pt.gather_owned(dist, w, bands, rank,
                             Pt.grid_view(Xd_loc, wl)[:, :, b.lat0 - b.lo:b.lat1 - b.lo])
        # reverse pass: the seed dL/dX^a on the owned rows only
        _, Wg = loss_mean_analysis(Xa, inp.truth)
        Wl = Pt.grid_view(Wg, w)[:, :, b.lo:b.hi].copy()
        Wl[:, :, :b.lat0 - b.lo] = 0.0
        Wl[:, :, b.lat1 - b.lo:] = 0.0
        _, Xb_bar_l, y_bar_l, R_bar_l = analysis_with_gradient(
            wl, Xl, inp.y[pos], inp.R[pos], inp.Z[:, pos], lab, Wl.reshape(w.N, -1))
        Xb_bar_band = Pt.halo_reduce(dist, w, bands, rank, Pt.grid_view(Xb_bar_l, wl))
        Xb_bar = Pt.gather_owned(dist, w, bands, rank, Xb_bar_band)
        y_bar = Pt.obs_reduce(dist, w, bands, rank, inp.obs_idx, pos, y_bar_l)
        R_bar = Pt.obs_reduce(dist, w, bands, rank, inp.obs_idx, pos, R_bar_l)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), Xa=Xa, Xd=Xd, Xb_bar=Xb_bar, y_bar=y_bar,
                 R_bar=R_bar, scatter_ok=scatter_ok, lat0=b.lat0, lat1=b.lat1, lo=b.lo,
                 hi=b.hi)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_band_plan_covers_the_grid_once():
    from paper_1606_00807_gb300 import partition as Pt
    from synthetic import WORKLOADS
    w = WORKLOADS["t63_192x96x29_n80_r2"]
    for world in (1, 2, 3, 4, 8):
        bands = Pt.band_plan(w, world)
        assert bands[0].lat0 == 0 and bands[-1].lat1 == w.nlat
        for a, c in zip(bands, bands[1:]):
            assert a.lat1 == c.lat0 and a.lat1 % w.sub_lat == 0
        for bb in bands:   # the local grid starts on a tile boundary, one tile row of halo
            assert bb.lo % w.sub_lat == 0 and bb.lat0 - bb.lo <= w.sub_lat
            assert bb.hi - bb.lat1 <= w.sub_lat and w.sub_lat >= w.r
    with pytest.raises(ValueError):
        Pt.band_plan(w, 9)


def test_two_ranks_reproduce_the_single_process_analysis_and_gradient(tmp_path):
    import oracle as O
    from oracle.adjoint import analysis_with_gradient, loss_mean_analysis
    from synthetic import WORKLOADS, make_inputs
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    w = WORKLOADS[WORKLOAD]
    inp = make_inputs(w)
    Xa_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx)
    Xd_ref = O.assimilate(w, inp.Xb, inp.y, inp.R, inp.Z, inp.obs_idx, form="dual")
    _, W = loss_mean_analysis(Xa_ref, inp.truth)
    _, Xb_bar, y_bar, R_bar = analysis_with_gradient(w, inp.Xb, inp.y, inp.R, inp.Z,
                                                     inp.obs_idx, W)
    for k in range(world):
        assert bool(r[k]["scatter_ok"])
        assert O.rel_err(r[k]["Xa"], Xa_ref) < 1e-12
        assert O.rel_err(r[k]["Xd"], Xd_ref) < 1e-12
        assert O.rel_err(r[k]["Xb_bar"], Xb_bar) < 1e-10
        assert O.rel_err(r[k]["y_bar"], y_bar) < 1e-10
        assert O.rel_err(r[k]["R_bar"], R_bar) < 1e-10
    # the bands split the sub-domain rows, halos of one tile row
    assert int(r[0]["lat1"]) == int(r[1]["lat0"])
