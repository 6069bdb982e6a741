"""Host-side split of the symmetric pair list across ranks.

The pair solves of Sec. 3 are independent; a multi-GPU run gives each rank a
contiguous, count-balanced range of the upper-triangular pair list
(kx_vx_apply_pairs) and sums the partial Vx psi and E_x with one reduce.
"""


def n_pairs(n_orb: int) -> int:
    return n_orb * (n_orb + 1) // 2


def pair_range(n_orb: int, rank: int, world: int):
    """[begin, end) of the symmetric pair list owned by `rank` of `world` ranks."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    P = n_pairs(n_orb)
    return (rank * P) // world, ((rank + 1) * P) // world


ORB_BLOCK = 4  # orbitals per block of the library's pair enumeration


def pair_list(n_orb: int):
    """The library's enumeration of the unordered pairs (i <= j): orbitals in
    blocks of ORB_BLOCK, block pairs (I, J), I <= J, row-major; inside a
    diagonal block i <= j row-major, inside an off-diagonal block all (i, j)."""
    out = []
    nb = (n_orb + ORB_BLOCK - 1) // ORB_BLOCK
    for IB in range(nb):
        for JB in range(IB, nb):
            I = range(IB * ORB_BLOCK, min(n_orb, (IB + 1) * ORB_BLOCK))
            J = range(JB * ORB_BLOCK, min(n_orb, (JB + 1) * ORB_BLOCK))
            for i in I:
                for j in J:
                    if IB != JB or j >= i:
                        out.append((i, j))
    return out


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
