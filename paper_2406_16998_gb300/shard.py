"""Host-side split of the pair solves across ranks.

The pair solves of Sec. 3 are independent.  Two splits are provided:

* contiguous, count-balanced ranges of the upper-triangular pair list
  (kx_vx_apply_pairs), summed with one all-reduce of the full Vx psi;
* the two-dimensional block-cyclic split: orbital blocks of four, block pairs
  (I, J), I <= J, owned by rank (I mod pr) pc + (J mod pc) of a pr x pc
  process grid (kx_vx_apply_block_pairs computes a rank's share); the partial
  Vx psi are combined by one reduce-scatter over contiguous orbital rows (each
  rank ends with the rows it owns) and E_x by a scalar all-reduce.  This
  replaces the paper's band/domain decomposition with its cyclic exchanges
  and all-to-alls (Sec. 4).
"""
import math


def n_pairs(n_orb: int) -> int:
    return n_orb * (n_orb + 1) // 2


def pair_range(n_orb: int, rank: int, world: int):
    """[begin, end) of the symmetric pair list owned by `rank` of `world` ranks."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    P = n_pairs(n_orb)
    return (rank * P) // world, ((rank + 1) * P) // world


ORB_BLOCK = 4  # orbitals per block of the library's pair enumeration


def n_blocks(n_orb: int) -> int:
    return (n_orb + ORB_BLOCK - 1) // ORB_BLOCK


def leading_columns(nb: int) -> int:
    """The fewest leading block columns that hold 15% of the block pairs."""
    want = (15 * (nb * (nb + 1) // 2) + 99) // 100
    jc = 1
    while jc < nb and jc * (jc + 1) // 2 < want:
        jc += 1
    return jc


def block_pairs(n_orb: int):
    """The library's order of the orbital block pairs (I, J), I <= J: those of the
    leading columns J < jc column-major (J = 0 .. jc-1, I = 0 .. J), then the rest
    row-major (I = 0 .. nb-1, J = max(I, jc) .. nb-1)."""
    nb = n_blocks(n_orb)
    jc = leading_columns(nb)
    return ([(I, J) for J in range(jc) for I in range(J + 1)] +
            [(I, J) for I in range(nb) for J in range(max(I, jc), nb)])


def pair_list(n_orb: int):
    """The library's enumeration of the unordered pairs (i <= j): orbitals in
    blocks of ORB_BLOCK, block pairs in the order of block_pairs; inside a
    diagonal block i <= j row-major, inside an off-diagonal block all (i, j)."""
    return pairs_of_block_pairs(n_orb, block_pairs(n_orb))


def pair_at(n_orb: int, k: int):
    """(i, j) of entry k of the library's pair enumeration."""
    return pair_list(n_orb)[k]


def kpoint_blocks(n_kpt: int):
    """The k-point pair blocks (k, q), q >= k, in the order kx_vx_kpoints solves
    them; the block (k, q) serves Vx psi_k and, read conjugated, Vx psi_q."""
    return [(k, q) for k in range(n_kpt) for q in range(k, n_kpt)]


def kpoint_block_range(n_kpt: int, rank: int, world: int):
    """[begin, end) of kpoint_blocks owned by `rank` of `world` ranks (count-balanced;
    the partial Vx psi of the ranks add up to the whole)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    B = n_kpt * (n_kpt + 1) // 2
    return (rank * B) // world, ((rank + 1) * B) // world


# ------------------------------------------------- two-dimensional block-cyclic split
def process_grid(world: int):
    """(pr, pc), pr * pc = world, pr the largest divisor of world <= sqrt(world)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    pr = max(d for d in range(1, int(math.isqrt(world)) + 1) if world % d == 0)
    return pr, world // pr


def block_owner(I: int, J: int, world: int) -> int:
    """Rank owning block pair (I, J) in the block-cyclic split."""
    pr, pc = process_grid(world)
    return (I % pr) * pc + (J % pc)


def rank_block_pairs(n_orb: int, rank: int, world: int):
    """The block pairs of `rank` (row-major order)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return [bp for bp in block_pairs(n_orb) if block_owner(bp[0], bp[1], world) == rank]


def pairs_of_block_pairs(n_orb: int, bps):
    """The (i, j) pairs of the block pairs `bps`, in the library's order inside a
    block pair (diagonal blocks: i <= j)."""
    out = []
    for IB, JB in bps:
        I = range(IB * ORB_BLOCK, min(n_orb, (IB + 1) * ORB_BLOCK))
        J = range(JB * ORB_BLOCK, min(n_orb, (JB + 1) * ORB_BLOCK))
        for i in I:
            for j in J:
                if IB != JB or j >= i:
                    out.append((i, j))
    return out


def rows_per_rank(n_orb: int, world: int) -> int:
    return (n_orb + world - 1) // world


def row_range(n_orb: int, rank: int, world: int):
    """[begin, end) of the orbital rows of Vx psi that `rank` ends with."""
    r = rows_per_rank(n_orb, world)
    return min(n_orb, rank * r), min(n_orb, (rank + 1) * r)


def reduce_scatter_rows(partial, world: int, group=None):
    """Sum of every rank's partial Vx psi (an (n_orb, N) tensor on each rank),
    returned as this rank's rows row_range(n_orb, rank, world): one
    reduce-scatter over row chunks of rows_per_rank rows (the last chunk
    padded with zero rows)."""
    import torch
    import torch.distributed as dist
    n_orb, N = partial.shape
    r = rows_per_rank(n_orb, world)
    if r * world != n_orb:
        pad = torch.zeros((r * world - n_orb, N), dtype=partial.dtype, device=partial.device)
        partial = torch.cat([partial, pad])
    out = torch.empty((r, N), dtype=partial.dtype, device=partial.device)
    dist.reduce_scatter_tensor(out, partial.contiguous(), group=group)
    rank = dist.get_rank(group)
    a, b = row_range(n_orb, rank, world)
    return out[: b - a]


def sharded_exchange(partial_fn, n_orb: int, rank: int, world: int, group=None):
    """One rank's part of the block-cyclic split.  partial_fn(block_pairs) returns
    (partial Vx psi as an (n_orb, N) tensor, partial E_x as a float) over those
    block pairs (kx_vx_apply_block_pairs on a GPU); returns (this rank's rows of
    Vx psi, E_x of the whole system)."""
    import torch
    import torch.distributed as dist
    vx_part, e_part = partial_fn(rank_block_pairs(n_orb, rank, world))
    rows = reduce_scatter_rows(vx_part, world, group)
    e = torch.tensor([float(e_part)], dtype=torch.float64, device=vx_part.device)
    dist.all_reduce(e, group=group)
    return rows, float(e.item())


def block_cyclic_bytes(n_orb: int, N: int, world: int, elem: int = 8):
    """Bytes each rank sends (and receives) in the ring reduce-scatter of the
    partial Vx psi, the size of its result rows, and of an all-gather of psi."""
    r = rows_per_rank(n_orb, world)
    total = r * world * N * elem
    return {"reduce_scatter_per_rank": total * (world - 1) // world, "result_rows_per_rank": r * N * elem,
            "psi_all_gather_per_rank": total * (world - 1) // world}
