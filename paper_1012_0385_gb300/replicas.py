"""Replicas: one process per GPU, each on its own disjoint range of samples.

Every sample draws its random numbers from Philox counters keyed by its
global index (``first_sample`` + local index), so rank r running samples
[r*S, (r+1)*S) produces exactly the samples that one run over N*S samples
would produce for that range.  The ranks therefore exchange nothing while
they sweep; the paper's multi-GPU runs likewise split independent samples
(Sec. 2.4).  The only collectives are the timing reduction (the maximum
over ranks of the elapsed time) and, for a caller that wants one table, a
gather of the int64 height sums in rank order, which is exact.

These helpers take the ``torch.distributed`` module and work with any
backend (NCCL between GPUs, gloo on the CPU).
"""
from __future__ import annotations

import numpy as np


def sample_range(rank: int, world: int, samples_per_rank: int) -> tuple[int, int]:
    """(first global sample, number of samples) of `rank` in a run of `world`
    replicas with `samples_per_rank` samples each (weak scaling)."""
    if world < 1 or not 0 <= rank < world or samples_per_rank < 1:
        raise ValueError(f"bad replica layout rank={rank} world={world} samples={samples_per_rank}")
    return rank * samples_per_rank, samples_per_rank


def _active(dist) -> bool:
    return dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(values, dist=None, device="cpu") -> list[float]:
    """Element-wise maximum of per-rank float values (e.g. elapsed ms)."""
    vals = [float(v) for v in values]
    if not _active(dist):
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def gather_samples(table: np.ndarray, dist=None, device="cpu", axis: int = 1) -> np.ndarray:
    """Concatenate every rank's int64/uint64 table along the sample axis, in
    rank order (all ranks must pass tables of the same shape).  Unsigned
    tables travel as their int64 bit pattern and come back unchanged."""
    if not _active(dist):
        return table
    import torch

    unsigned = table.dtype == np.uint64
    if table.dtype not in (np.int64, np.uint64):
        raise TypeError(f"gather_samples takes 64-bit integer tables, not {table.dtype}")
    src = np.ascontiguousarray(table).view(np.int64)
    t = torch.from_numpy(src.copy()).to(device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    out = np.concatenate([p.cpu().numpy() for p in parts], axis=axis)
    return out.view(np.uint64) if unsigned else out


def throughput(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    if max_ms <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank_step * steps * world / (max_ms / 1000.0)
