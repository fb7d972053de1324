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


class OraclePlan:
    """CPU stand-in for api.Plan in the host-logic tests: the same translate_average
    signature and return types, computed by the oracle."""

    def __init__(self, dims):
        self.dims = dims

    def translate_average(self, phase, phases, c0, b, shifts, E=(0.0,) * 6, tol=1e-6, maxit=10000):
        from oracle import bfcs_oracle as O
        avg, hits, infos = O.translate_average(phase.numpy(), phases, c0, b.numpy(), shifts, E, tol, maxit)
        return torch.from_numpy(np.ascontiguousarray(avg)), torch.from_numpy(hits.astype(np.int32)), infos


def _product_rank(rank, world, port, result_path, nshift):
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
        shifts = [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 3, 3), (5, 1, 7)][:nshift]
        avg, hits, infos = D.translate_average(OraclePlan(dims), torch.from_numpy(ph), phases, c0,
                                               torch.from_numpy(b), shifts, tol=1e-11, maxit=2000)
        lo, hi = D.shard(len(shifts), rank, world)
        assert len(infos) == hi - lo
        ref_avg, ref_hits, _ = O.translate_average(ph, phases, c0, b, shifts, tol=1e-11, maxit=2000)
        err = float(np.linalg.norm(avg.numpy() - ref_avg) / np.linalg.norm(ref_avg))
        same_hits = bool(np.array_equal(hits.numpy(), ref_hits))
        with open(f"{result_path}.{rank}", "w") as f:
            f.write(f"{err} {int(same_hits)} {hi - lo}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nshift", [(2, 5), (3, 2)])
def test_product_translate_average_over_gloo_ranks(tmp_path, world, nshift):
    """distributed.translate_average itself (sharding, the local solve through the
    plan's translate_average, the all-reduce of the sums and hit counts) on gloo
    ranks with a CPU stand-in plan; with 3 ranks and 2 shifts one rank owns no
    shift and contributes zeros.  Every rank gets the full average."""
    path = str(tmp_path / "result")
    mp.start_processes(_product_rank, args=(world, _free_port(), path, nshift), nprocs=world, join=True,
                       start_method="spawn")
    owned = 0
    for r in range(world):
        err, same, n = open(f"{path}.{r}").read().split()
        assert float(err) < 1e-13 and same == "1", r
        owned += int(n)
    assert owned == nshift


def _dying_rank(rank, world, port, result_path):
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)                                  # leaves between steps, before the exchange
    from oracle import bfcs_oracle as O
    from paper_2601_00822_gb300 import workloads as W
    dims = (8, 8, 8)
    phases = [(1.0, 0.5), (10.0, 5.0)]
    ph = O.phase_map(dims, (8, 8, 8), np.asarray([W.sphere_row(4, 4, 4, 2.5)], dtype=np.int32))
    b = O.body_force(dims, (4.0, 4.0, 4.0), 3.0)
    t0 = time.monotonic()
    outcome = "returned"
    try:
        D.translate_average(OraclePlan(dims), torch.from_numpy(ph), phases, W.reference_medium(phases),
                            torch.from_numpy(b), [(0, 0, 0), (1, 0, 0)], tol=1e-8, maxit=500)
    except Exception as e:                           # the collective reports the missing peer
        outcome = type(e).__name__
    with open(result_path, "w") as f:
        f.write(f"{outcome} {time.monotonic() - t0:.3f}")
    os._exit(0)


def test_a_rank_that_leaves_gives_an_error_not_a_hang(tmp_path):
    """Failure detection on the host: rank 1 exits before the all-reduce of the
    sharded averaging; rank 0's exchange ends with an error within the process
    group's timeout instead of waiting forever."""
    path = str(tmp_path / "outcome.txt")
    ctx = mp.start_processes(_dying_rank, args=(2, _free_port(), path), nprocs=2, join=False,
                             start_method="spawn")
    import time
    t0 = time.monotonic()
    while not ctx.join(timeout=1.0):
        assert time.monotonic() - t0 < 120, "rank 0 did not return"
    outcome, secs = open(path).read().split()
    assert outcome != "returned" and float(secs) < 60.0, (outcome, secs)


def test_bench_relaunches_itself_with_one_process_per_gpu():
    """bench.py --gpus N outside a launcher re-executes itself under
    torch.distributed.run with N processes on 127.0.0.1 and the same arguments."""
    import importlib.util
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cmd = bench.torchrun_argv(4, ["--gpus", "4", "--steps", "3"], 29511)
    assert cmd[:3] == [sys.executable, "-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29511"
    assert cmd[-4:] == ["--gpus", "4", "--steps", "3"] and cmd[-5].endswith("bench.py")
