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
N_ALL = slice(52, 54)      # ledger slots of the collisions and flights of every pass


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
    tallies of the last pass, whose ledger counts the collisions and flights
    of both passes in its all-pass slots as karl_run does (identical on every
    rank)."""
    a, b = shard_range(prims.n, rank, world)
    mine = prims.slice(a, b - a)
    t = run_pass(mine, seed, 1, None, a, prims.n_decays)
    if n_passes == 2:
        time1 = _allreduce_sum(t["time_fx"]) if world > 1 else t["time_fx"]
        all1 = t["ledger"][N_ALL].copy()
        t = run_pass(mine, seed, 2, time1, a, prims.n_decays)
        t["ledger"][N_ALL] += all1          # collisions and flights of both passes
    out = {}
    for k in RAW_KEYS:
        out[k] = _allreduce_sum(t[k]) if world > 1 else t[k]
    return out


def run_cycles_sharded(run_cycle: Callable, prims, seed: int, n_cycles: int, rank: int,
                       world: int) -> Dict[str, np.ndarray]:
    """The continuous field update (Sec. 3.6) split over `world` ranks: every
    cycle's primary-id range [c n / C, (c+1) n / C) is split over the ranks,
    each rank runs its part with the fields of the summed tallies of the
    cycles before (the same on every rank), and one integer all-reduce per
    cycle adds the cycle's raw tallies -- the paper's synchronisation step
    after each cycle.  ``run_cycle(prims_slice, seed, field_time_in,
    field_recomb_in, field_decays, pid_offset)`` is the per-rank cycle
    (``karl.Context.run_cycle`` on a GPU).  Returns the raw tallies summed
    over all cycles and ranks (identical on every rank)."""
    n = prims.n
    tot: Dict[str, np.ndarray] = {}
    for c in range(n_cycles):
        lo, hi = c * n // n_cycles, (c + 1) * n // n_cycles
        if hi <= lo:
            continue
        a, b = shard_range(hi - lo, rank, world)
        a, b = lo + a, lo + b
        first = not tot
        t = run_cycle(prims.slice(a, b - a), seed, None if first else tot["time_fx"],
                      None if first else tot["recomb"], prims.n_decays * lo / n, a)
        for k in RAW_KEYS:
            s = _allreduce_sum(t[k]) if world > 1 else t[k]
            tot[k] = s if k not in tot else tot[k] + s
    return tot


ORBIT_RAW_KEYS = ("spectrum", "time_z", "time_r", "cross_pos", "cross_neg", "rcross_out",
                  "rcross_in", "wall", "ledger", "chan_count")


def run_orbit_sharded(run_orbit: Callable, prims, seed: int, rank: int,
                      world: int) -> Dict[str, np.ndarray]:
    """The full-orbit run (one pass, no fields fed back) split over `world`
    ranks by primary-id ranges: histories are independent and their random
    streams keyed by primary id, so one integer all-reduce of the raw
    tallies gives the single run's tallies bit for bit; the FP64 energy
    ledger is summed as well (equal to rounding).  ``run_orbit(prims_slice,
    seed)`` is the per-rank run (``karl.Context.run_orbit`` on a GPU); the
    slice carries its primary-id offset."""
    a, b = shard_range(prims.n, rank, world)
    mine = type(prims)(*(getattr(prims, k)[a:b].copy() for k in
                         ("x_m", "y_m", "z_m", "e_ev", "mu", "phi", "species")),
                       pid_offset=int(prims.pid_offset) + a)
    t = run_orbit(mine, seed)
    out = {k: _allreduce_sum(t[k]) if world > 1 else t[k] for k in ORBIT_RAW_KEYS}
    if world > 1:
        import torch
        import torch.distributed as dist
        e = torch.from_numpy(np.ascontiguousarray(t["energy"], np.float64).copy())
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        out["energy"] = e.numpy()
    else:
        out["energy"] = t["energy"]
    return out
