"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the way
torchrun launches one process per GPU), each with its own shard of the
cell sequence, the barrier around the timed region and the maximum of the
ranks' times."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        slowest = bench.max_over_ranks(10.0 + rank, world)
        w = bench.make_workload("mech22", cells=8, shard=rank)
        m = bench.make_workload("mixed", cells=2, shard=rank)
        bench.barrier(world)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), slowest=slowest, y0=w["y0"],
                 e0=m["e0"], ym=m["y0_mech"])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_cells_and_take_the_slowest_time(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    assert all(float(x["slowest"]) == 11.0 for x in r)
    full = bench.make_workload("mech22", cells=16)
    np.testing.assert_array_equal(np.concatenate([r[0]["y0"], r[1]["y0"]]), full["y0"])
    mixed = bench.make_workload("mixed", cells=4)
    np.testing.assert_array_equal(np.concatenate([r[0]["e0"], r[1]["e0"]]), mixed["e0"][:1024])
    np.testing.assert_array_equal(np.concatenate([r[0]["ym"], r[1]["ym"]]), mixed["y0_mech"][:4])


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.shard_cells(1024, 3) == 3072
