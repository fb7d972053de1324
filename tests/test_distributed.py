"""The sharded translated averaging's host logic on CPU: two gloo ranks each
average their block of shifts (with the oracle standing in for the GPU solve)
and combine; the result equals the single-process average over all shifts."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_00822_gb300 import distributed as D


def test_shard_covers_every_item_once():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                lo, hi = D.shard(n, r, world)
                got += list(range(lo, hi))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import bfcs_oracle as O
        from paper_2601_00822_gb300 import workloads as W
        dims = (8, 8, 8)
        phases = [(1.0, 0.5), (10.0, 5.0)]
        c0 = W.reference_medium(phases)
        ph = O.phase_map(dims, (8, 8, 8), np.asarray([W.sphere_row(4, 4, 4, 2.5)], dtype=np.int32))
        b = O.body_force(dims, (4.0, 4.0, 4.0), 3.0)
        shifts = [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 3, 3), (5, 1, 7)]
        lo, hi = D.shard(len(shifts), rank, world)
        avg, hits, _ = O.translate_average(ph, phases, c0, b, shifts[lo:hi], tol=1e-11, maxit=2000)
        g_avg, g_hits = D.combine(torch.from_numpy(np.ascontiguousarray(avg)), torch.from_numpy(hits.astype(np.int32)),
                                  hi - lo, len(shifts))
        if rank == 0:
            ref_avg, ref_hits, _ = O.translate_average(ph, phases, c0, b, shifts, tol=1e-11, maxit=2000)
            err = float(np.linalg.norm(g_avg.numpy() - ref_avg) / np.linalg.norm(ref_avg))
            same_hits = bool(np.array_equal(g_hits.numpy(), ref_hits))
            with open(result_path, "w") as f:
                f.write(f"{err} {int(same_hits)}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_full_average(tmp_path):
    world = 2
    path = str(tmp_path / "result.txt")
    mp.start_processes(_rank, args=(world, _free_port(), path), nprocs=world, join=True, start_method="spawn")
    err, same = open(path).read().split()
    assert float(err) < 1e-13 and same == "1"
