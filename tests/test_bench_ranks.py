"""The benchmark's multi-rank host logic on CPU (gloo, two ranks).

bench.py runs one independent instance per GPU (weak scaling, no data-path
collective): each rank builds its own problem (the point source moved by
rank), and the timing is reduced over ranks (max of the times, sum of the
point updates).  These tests run that logic with the gloo backend on two CPU
processes; the reference arm prints on rank 0 only.
"""
import contextlib
import io
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench as b
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, _ = b.make_workload("2d_const_101", rank)
    t = 1.5 + rank                                   # this rank's "time"
    ups = float(np.prod(p.n)) * (rank + 1)
    tmax = b.all_reduce_scalar(t, dist.ReduceOp.MAX, world, "cpu")
    usum = b.all_reduce_scalar(ups, dist.ReduceOp.SUM, world, "cpu")
    dist.barrier()
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), F=p.F, c=p.c_cell, tmax=tmax, usum=usum)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_build_independent_instances(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    n = np.prod(r[0]["F"].shape)
    for k in range(world):
        assert float(r[k]["tmax"]) == 2.5                  # max over ranks
        assert float(r[k]["usum"]) == float(n) * 3         # sum over ranks
    assert np.array_equal(r[0]["c"], r[1]["c"])            # same model ...
    assert not np.array_equal(r[0]["F"], r[1]["F"])        # ... its own source per rank
    assert np.abs(r[0]["F"]).sum() == np.abs(r[1]["F"]).sum()


def test_single_rank_reduction_is_identity():
    assert bench.all_reduce_scalar(3.25, None, 1, "cpu") == 3.25


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args([])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
