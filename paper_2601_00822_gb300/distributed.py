"""Translated averaging (Eqs. 3.3-3.6) sharded over ranks, one GPU per rank.

The shifts chi_m are split into contiguous blocks, one per rank; each rank
runs bfcs_translate_average on its block, turns its averages back into FP64
sums (average x number of local shifts), and one all-reduce of the 30 x N
sums and the N hit counts gives every rank the averages over all shifts.
This is the only exchange of the path; a single solve is never split.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [lo, hi) of n items owned by `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    return n * rank // world, n * (rank + 1) // world


def _all_reduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    if dist.get_backend(group) == "nccl" or not t.is_cuda:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t
    host = t.cpu()                      # gloo reduces host tensors
    dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
    t.copy_(host)
    return t


def combine(avg_local: torch.Tensor, hits_local: torch.Tensor, n_local: int, n_total: int, group=None):
    """Global averages and hit counts from every rank's local averages over
    its n_local shifts (n_local = 0: the rank contributes zeros)."""
    if n_total < 1:
        raise ValueError("no shifts")
    sums = avg_local.to(torch.float64) * float(n_local)
    hits = hits_local.to(torch.int64)
    _all_reduce_sum(sums, group)
    _all_reduce_sum(hits, group)
    return sums / float(n_total), hits.to(torch.int32)


def translate_average(plan, phase, phases, c0, b, shifts, E=(0.0,) * 6, tol=1e-6, maxit=10000, group=None):
    """bfcs_translate_average over all ranks of `group`: returns (avg (30, nz, ny, nx)
    float64, hits (nz, ny, nx) int32, this rank's solve infos)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    shifts = [tuple(int(v) for v in s) for s in shifts]
    lo, hi = shard(len(shifts), rank, world)
    nx, ny, nz = plan.dims
    if hi > lo:
        avg, hits, infos = plan.translate_average(phase, phases, c0, b, shifts[lo:hi], E=E, tol=tol, maxit=maxit)
    else:
        avg = torch.zeros((30, nz, ny, nx), dtype=torch.float64, device=phase.device)
        hits = torch.zeros((nz, ny, nx), dtype=torch.int32, device=phase.device)
        infos = []
    avg, hits = combine(avg, hits, hi - lo, len(shifts), group)
    return avg, hits, infos
