"""Run split over ranks: primary-id ranges per rank, one exchange per pass.

Histories are independent within a pass, so each rank follows a contiguous
range of primary ids; the only data exchanged is the integer sum of the raw
tallies (Sec. 3.6: the paper's ranks add their density fields, times,
currents and loggers).  Before pass 2 every rank needs the pass-1 time tally
of the whole run to build the same recombination target fields; after the
last pass the raw tallies are summed.  Tallies are u64 fixed point, so the
sums are exact and the result equals a single run bit for bit.

``run_pass(prims_slice, seed, pass_index, field_time_in, pid_offset, n_decays)``
is the per-rank pass (``karl.Context.run_pass`` on a GPU).  The collective is
``torch.distributed.all_reduce`` on int64 views of the u64 arrays (two's
complement addition is the same bit pattern).
"""
from __future__ import annotations

from typing import Callable, Dict

import numpy as np

RAW_KEYS = ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count")


def shard_range(n: int, rank: int, world: int):
    """Contiguous primary-id range [a, b) of a rank."""
    a = n * rank // world
    b = n * (rank + 1) // world
    return a, b


def _allreduce_sum(arr: np.ndarray) -> np.ndarray:
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy().view(arr.dtype).reshape(arr.shape)


def run_sharded(run_pass: Callable, prims, seed: int, n_passes: int, rank: int,
                world: int) -> Dict[str, np.ndarray]:
    """All passes of a run split over `world` ranks; returns the summed raw
    tallies of the last pass (identical on every rank)."""
    a, b = shard_range(prims.n, rank, world)
    mine = prims.slice(a, b - a)
    t = run_pass(mine, seed, 1, None, a, prims.n_decays)
    if n_passes == 2:
        time1 = _allreduce_sum(t["time_fx"]) if world > 1 else t["time_fx"]
        t = run_pass(mine, seed, 2, time1, a, prims.n_decays)
    out = {}
    for k in RAW_KEYS:
        out[k] = _allreduce_sum(t[k]) if world > 1 else t[k]
    return out
