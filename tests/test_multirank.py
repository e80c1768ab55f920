"""World-size-2 gloo ranks on CPU: the sharded run (primary-id ranges, one
integer all-reduce per pass) equals a single run bit for bit.  The per-rank
pass is the oracle here; on GPUs it is karl.Context.run_pass, which
tests/test_gpu_parity.py checks for shard additivity on one device."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2503_10263_gb300 import inputs, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, prims = inputs.config2(n_decays=150, seed=7, column_m2=2e21, length=4.0, nz=100)

    def run_pass(p, seed, pass_index, field, pid_offset, n_decays):
        return oracle.run_pass(prob, p, seed, pass_index, field_time_in=field,
                               pid_offset=pid_offset, n_decays=n_decays)

    t = shard.run_sharded(run_pass, prims, seed=13, n_passes=2, rank=rank, world=world)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **t)
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_single_run(tmp_path):
    oracle.build()
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    prob, prims = inputs.config2(n_decays=150, seed=7, column_m2=2e21, length=4.0, nz=100)
    full = oracle.run(prob, prims, seed=13)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    for k in shard.RAW_KEYS:
        np.testing.assert_array_equal(r0[k], r1[k], err_msg=k)
        np.testing.assert_array_equal(r0[k], full[k], err_msg=k)


def _cycle_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, prims = _cycled_problem()

    def run_cycle(p, seed, field, rec, decays, pid_offset):
        return oracle.run_cycle(prob, p, seed, field, rec, decays, pid_offset=pid_offset)

    t = shard.run_cycles_sharded(run_cycle, prims, seed=17, n_cycles=3, rank=rank, world=world)
    np.savez(os.path.join(out_dir, f"cyc{rank}.npz"), **t)
    dist.destroy_process_group()


def _cycled_problem():
    prob, prims = inputs.config2(n_decays=150, seed=8, column_m2=2e21, length=4.0, nz=100)
    prob.activity_bq *= 1e9                                 # fields that matter
    return prob, prims


def test_two_gloo_ranks_cycles_equal_single_run(tmp_path):
    # the continuous field update split over ranks, one all-reduce per cycle
    oracle.build()
    world = 2
    mp.start_processes(_cycle_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    prob, prims = _cycled_problem()
    full = oracle.run_cycles(prob, prims, 17, 3)
    r0 = np.load(tmp_path / "cyc0.npz")
    r1 = np.load(tmp_path / "cyc1.npz")
    assert int(np.sum(full["recomb"])) > 0
    for k in shard.RAW_KEYS:
        np.testing.assert_array_equal(r0[k], r1[k], err_msg=k)
        np.testing.assert_array_equal(r0[k], full[k], err_msg=k)


def test_shard_ranges_cover_all_primaries():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            rs = [shard.shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))


def _orbit_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, orb, pr = inputs.orbit_config(n_decays=40, seed=5)

    def run_orbit(p, seed):
        return oracle.orbit_run(prob, orb, p, seed=seed)

    t = shard.run_orbit_sharded(run_orbit, pr, seed=21, rank=rank, world=world)
    np.savez(os.path.join(out_dir, f"orbit{rank}.npz"), **t)
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_single_orbit_run(tmp_path):
    """The full-orbit form shards the same way: two ranks' summed tallies
    equal the single run bit for bit (the energy ledger to rounding)."""
    oracle.build()
    world = 2
    mp.start_processes(_orbit_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    prob, orb, pr = inputs.orbit_config(n_decays=40, seed=5)
    full = oracle.orbit_run(prob, orb, pr, seed=21, n_threads=2)
    r0 = np.load(tmp_path / "orbit0.npz")
    r1 = np.load(tmp_path / "orbit1.npz")
    for k in shard.ORBIT_RAW_KEYS:
        np.testing.assert_array_equal(r0[k], r1[k], err_msg=k)
        np.testing.assert_array_equal(r0[k], full[k], err_msg=k)
    np.testing.assert_allclose(r0["energy"], full["energy"], rtol=1e-12, atol=1e-9)
