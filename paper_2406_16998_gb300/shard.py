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


def pair_at(n_orb: int, k: int):
    """(i, j) of entry k of the row-major upper-triangular list (i <= j)."""
    i = 0
    row = n_orb
    while k >= row:
        k -= row
        i += 1
        row -= 1
    return i, i + k
