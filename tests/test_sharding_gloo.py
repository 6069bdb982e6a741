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


# ---------------------------------------------------------------- k-point blocks
K_SYS = dict(n=(8, 10, 9), h=(0.5, 0.45, 0.5), bc=(1, 1, 0), kernel=0, n_orb=2, n_centres=3, seed=81)


def _block_partial(base, theta, wk, psi, occ, blocks):
    """Vx psi (all k-points) from the given blocks only: the block (k, q) adds q's
    bands to Vx psi_k and, for q > k, k's bands to Vx psi_q (oracle arithmetic on
    the two-k-point sub-problem with the target's own weight set to zero)."""
    n_kpt = psi.shape[0]
    out = np.zeros_like(psi)
    for k, q in blocks:
        if q == k:
            out[k] += oracle.vx_apply_kpoint(base, theta[[k]], wk[[k]], psi[[k]], occ[[k]], 0, psi[k])
            continue
        out[k] += oracle.vx_apply_kpoint(base, theta[[k, q]], np.array([0.0, wk[q]]), psi[[k, q]], occ[[k, q]], 0,
                                         psi[k])
        out[q] += oracle.vx_apply_kpoint(base, theta[[q, k]], np.array([0.0, wk[k]]), psi[[q, k]], occ[[q, k]], 0,
                                         psi[q])
    return out


def _kpoint_inputs():
    sysd = workloads.System(**K_SYS)
    theta, wk = workloads.kpoint_grid(sysd, (3, 1, 1))
    psi = workloads.make_bloch_orbitals(sysd, theta)
    occ = np.random.default_rng(3).uniform(0.4, 1.0, (len(wk), sysd.n_orb))
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    return sysd, base, theta, wk, psi, occ


def test_kpoint_block_range_covers_blocks_exactly():
    for n_kpt in (1, 2, 4, 9):
        B = len(shard.kpoint_blocks(n_kpt))
        assert B == n_kpt * (n_kpt + 1) // 2
        for world in (1, 2, 3, 8):
            ranges = [shard.kpoint_block_range(n_kpt, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == B
            assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))


def _kpoint_rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysd, base, theta, wk, psi, occ = _kpoint_inputs()
    a, b = shard.kpoint_block_range(len(wk), rank, world)
    part = _block_partial(base, theta, wk, psi, occ, shard.kpoint_blocks(len(wk))[a:b])
    t = torch.from_numpy(np.ascontiguousarray(part).view(np.float64).reshape(-1).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_kpoint_blocks_sum_to_full():
    """The k-point blocks split over two gloo ranks: the all-reduced partial
    Vx psi equals the oracle's Vx psi at every k-point, and so does E_x formed
    from it."""
    world = 2
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "sum.npy")
        mp.start_processes(_kpoint_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        got = np.load(out)
    sysd, base, theta, wk, psi, occ = _kpoint_inputs()
    vx, ex = oracle.vx_kpoints(base, theta, wk, psi, occ)
    got = got.view(np.complex128).reshape(vx.shape)
    assert np.max(np.abs(got - vx)) < 1e-12 * np.abs(vx).max()
    e = sum(0.5 * base.dV * wk[k] * occ[k, n] * np.vdot(psi[k][:, n], got[k][:, n]).real
            for k in range(len(wk)) for n in range(sysd.n_orb))
    assert abs(e - ex) < 1e-12 * abs(ex)


# ------------------------------------------------------ block-cyclic split + reduce-scatter
BC_SYS = dict(n=(10, 12, 14), h=(0.5, 0.45, 0.4), bc=(0, 1, 0), kernel=1, n_orb=11, n_centres=3, seed=79)


def test_block_cyclic_owners_partition_the_pairs():
    for n_orb in (1, 4, 11, 64, 256):
        allp = sorted(shard.pair_list(n_orb))
        for world in (1, 2, 3, 4, 6, 8):
            pr, pc = shard.process_grid(world)
            assert pr * pc == world and pr <= pc
            got = []
            for r in range(world):
                bps = shard.rank_block_pairs(n_orb, r, world)
                assert all(shard.block_owner(I, J, world) == r and I <= J for I, J in bps)
                got += shard.pairs_of_block_pairs(n_orb, bps)
            assert sorted(got) == allp
            rows = [shard.row_range(n_orb, r, world) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == n_orb
            assert all(rows[r][1] == rows[r + 1][0] for r in range(world - 1))


def _bc_rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysd = workloads.System(**BC_SYS)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)

    def partial(bps):  # this rank's block pairs with oracle arithmetic (the GPU call on a GPU rank)
        vx, ex = oracle.vx_apply(op, psi, pairs=shard.pairs_of_block_pairs(sysd.n_orb, bps))
        return torch.from_numpy(np.ascontiguousarray(vx.T)), ex

    rows, ex = shard.sharded_exchange(partial, sysd.n_orb, rank, world)
    a, b = shard.row_range(sysd.n_orb, rank, world)
    np.save(os.path.join(out_dir, f"rows{rank}.npy"), rows.numpy())
    np.save(os.path.join(out_dir, f"ex{rank}.npy"), np.array([ex, a, b]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_block_cyclic_reduce_scatter_gives_each_rank_its_rows(world):
    """Each rank computes its block pairs of the 2D block-cyclic split, one
    reduce-scatter leaves it the summed rows it owns, one scalar all-reduce
    gives E_x; together the rows are the oracle's full Vx psi."""
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_bc_rank_main, args=(world, _free_port(), d), nprocs=world, start_method="spawn")
        got = [(np.load(os.path.join(d, f"rows{r}.npy")), np.load(os.path.join(d, f"ex{r}.npy")))
               for r in range(world)]
    sysd = workloads.System(**BC_SYS)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    vx, ex = oracle.vx_apply(op, psi)
    full = np.concatenate([g[0] for g in got])
    assert full.shape == (sysd.n_orb, op.N)
    assert np.max(np.abs(full - vx.T)) < 1e-12 * np.abs(vx).max()
    for r, (rows, meta) in enumerate(got):
        assert (int(meta[1]), int(meta[2])) == shard.row_range(sysd.n_orb, r, world)
        assert abs(meta[0] - ex) < 1e-12 * abs(ex)
