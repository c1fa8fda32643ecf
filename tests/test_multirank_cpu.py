"""The multi-rank bench path on CPU: two `gloo` ranks (world size 2).

`bench.py --gpus N` runs one independent problem per rank (same shapes, own
seed, no exchange during the analysis) and reports every rank's cycles over
the slowest rank's time.  These tests run that host logic -- the per-rank
workload, the max over ranks and the whole-job rate -- in two spawned CPU
processes joined by a gloo process group on 127.0.0.1.
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


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from synthetic import WORKLOADS, make_inputs

        w = bench.rank_workload(WORKLOADS["tiny_32x16_n20_r2"], rank)
        inp = make_inputs(w, np.float64)
        # each rank's own timing; the job time is the slowest rank's
        ms = 10.0 + 5.0 * rank
        t_max = bench.slowest_rank(ms, world, torch.device("cpu"))
        rate = bench.job_rate(30, world, t_max / 1e3)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), seed=w.seed, n=w.n, N=w.N,
                 xb=inp.Xb[:2, :8], t_max=t_max, rate=rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_independent_problems_and_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # same shapes, different seeds and data: independent problems
    assert int(r[0]["n"]) == int(r[1]["n"]) and int(r[0]["N"]) == int(r[1]["N"])
    assert int(r[0]["seed"]) != int(r[1]["seed"])
    assert not np.array_equal(r[0]["xb"], r[1]["xb"])
    # every rank sees the slowest rank's time and the same whole-job rate
    for k in range(world):
        assert float(r[k]["t_max"]) == 15.0
        assert float(r[k]["rate"]) == pytest.approx(30 * world / 15e-3)


def test_single_rank_needs_no_process_group():
    import bench
    from synthetic import WORKLOADS

    w = WORKLOADS["tiny_32x16_n20_r2"]
    assert bench.rank_workload(w, 0) is w
    assert bench.slowest_rank(12.5, 1, None) == 12.5
    assert bench.job_rate(10, 1, 0.5) == 20.0
