"""The pair-list split a multi-GPU run would use, exercised with world-size-2
gloo ranks on the CPU: each rank sums its contiguous range of pair solves
(oracle arithmetic), one all-reduce combines the partial Vx psi and E_x, and the
result equals the unsplit computation."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from paper_2406_16998_gb300 import shard


def test_pair_range_covers_list_exactly():
    for n_orb in (1, 2, 5, 64):
        P = shard.n_pairs(n_orb)
        lst = shard.pair_list(n_orb)
        assert len(lst) == P and sorted(lst) == sorted(oracle.pair_list(n_orb, ordered=False))
        for world in (1, 2, 3, 8):
            ranges = [shard.pair_range(n_orb, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysd = workloads.System(n=(10, 12, 14), h=(0.5, 0.45, 0.4), bc=(0, 1, 0), kernel=1, n_orb=5, n_centres=3,
                            seed=77)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    a, b = shard.pair_range(sysd.n_orb, rank, world)
    pairs = shard.pair_list(sysd.n_orb)[a:b]
    vx, ex = oracle.vx_apply(op, psi, pairs=pairs)
    t = torch.from_numpy(np.concatenate([vx.reshape(-1), [ex]]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_split_sums_to_full():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "sum.npy")
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        got = np.load(out)
    sysd = workloads.System(n=(10, 12, 14), h=(0.5, 0.45, 0.4), bc=(0, 1, 0), kernel=1, n_orb=5, n_centres=3,
                            seed=77)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    vx, ex = oracle.vx_apply(op, psi)
    assert np.max(np.abs(got[:-1].reshape(vx.shape) - vx)) < 1e-12 * np.abs(vx).max()
    assert abs(got[-1] - ex) < 1e-12 * abs(ex)
