"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the exchange method itself: it only builds
grids, orbital sets and workload descriptions.  Orbitals are sums of s/p
Gaussian primitives on a uniform finite-difference grid (the kind of localized
functions the paper's molecules and bulk cells produce, Sec. 4), orthonormalised
by FP64 CholeskyQR2 under the quadrature inner product <a, b> = dV * sum(a * b).

Layout of every orbital block: a float64 array of shape (N, n_orb), N = n1*n2*n3,
grid index flattened with x1 fastest, then x2, then x3 (Sec. 3, frontal slices
B(:, :, k) are contiguous n1*n2 blocks).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

DIRICHLET = 0
PERIODIC = 1
UNSCREENED = 0
SCREENED = 1

HSE_OMEGA = 0.11  # bohr^-1


@dataclass(frozen=True)
class System:
    """One exchange problem: grid, boundary conditions, kernel and orbital recipe."""
    n: tuple            # (n1, n2, n3)
    h: tuple            # (h1, h2, h3) grid spacing in bohr
    bc: tuple           # per axis: DIRICHLET or PERIODIC
    kernel: int         # UNSCREENED or SCREENED
    n_orb: int
    n_centres: int      # "atom" centres the primitives sit on (0: each primitive its own)
    omega: float = HSE_OMEGA
    fd_order: int = 12
    seed: int = 1234
    name: str = ""

    @property
    def N(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def dV(self) -> float:
        return self.h[0] * self.h[1] * self.h[2]

    def lengths(self):
        """Box length per axis: (n+1)h for Dirichlet (zero values at x=0 and x=L), nh for periodic."""
        return tuple((self.n[a] + 1) * self.h[a] if self.bc[a] == DIRICHLET else self.n[a] * self.h[a]
                     for a in range(3))


def grid_coords(sys: System, axis: int) -> np.ndarray:
    """Coordinates of the unknowns along one axis: x_i=(i+1)h (Dirichlet), x_i=ih (periodic)."""
    n, h = sys.n[axis], sys.h[axis]
    i = np.arange(n, dtype=np.float64)
    return (i + 1.0) * h if sys.bc[axis] == DIRICHLET else i * h


def _axis_offsets(sys: System, axis: int, c: float) -> np.ndarray:
    x = grid_coords(sys, axis)
    d = x - c
    if sys.bc[axis] == PERIODIC:
        L = sys.n[axis] * sys.h[axis]
        d = (d + 0.5 * L) % L - 0.5 * L  # minimum image
    return d


def cholesky_qr2(psi: np.ndarray, dV: float) -> np.ndarray:
    """Orthonormalise columns under <a,b> = dV a.b with two CholeskyQR passes (FP64)."""
    for _ in range(2):
        G = dV * (psi.T @ psi)
        Lc = np.linalg.cholesky(G)
        psi = np.linalg.solve(Lc, psi.T).T  # psi <- psi Lc^{-T}
    return np.ascontiguousarray(psi)


def make_orbitals(sys: System, n_orb: int | None = None, seed: int | None = None) -> np.ndarray:
    """Seeded orbitals, shape (N, n_orb) float64, x1 fastest, dV-orthonormal.

    Each orbital is a sum of 3 primitives; each primitive is s-type exp(-a r^2) or
    p-type (x_ax - c_ax) exp(-a r^2) (50/50, axis uniform), exponent a ~ U[0.5, 2]
    bohr^-2, coefficient ~ N(0, 1).  Centres: for Dirichlet axes U[L/4, 3L/4], for
    periodic axes U[0, L) with minimum-image distances.
    """
    n_orb = sys.n_orb if n_orb is None else n_orb
    rng = np.random.default_rng(sys.seed if seed is None else seed)
    Ls = sys.lengths()
    n_c = sys.n_centres if sys.n_centres > 0 else 3 * n_orb
    lo = np.array([0.25 * Ls[a] if sys.bc[a] == DIRICHLET else 0.0 for a in range(3)])
    hi = np.array([0.75 * Ls[a] if sys.bc[a] == DIRICHLET else Ls[a] for a in range(3)])
    centres = rng.uniform(lo, hi, size=(n_c, 3))
    n1, n2, n3 = sys.n
    psi = np.zeros((sys.N, n_orb), dtype=np.float64)
    for i in range(n_orb):
        acc = np.zeros((n3, n2, n1), dtype=np.float64)
        for p in range(3):
            atom = int(rng.integers(n_c)) if sys.n_centres > 0 else 3 * i + p
            kind = int(rng.integers(2))
            ax = int(rng.integers(3))
            alpha = float(rng.uniform(0.5, 2.0))
            coef = float(rng.standard_normal())
            c = centres[atom]
            d = [_axis_offsets(sys, a, c[a]) for a in range(3)]
            g = [np.exp(-alpha * d[a] ** 2) for a in range(3)]
            if kind == 1:
                g[ax] = g[ax] * d[ax]
            acc += coef * (g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :])
        psi[:, i] = acc.reshape(-1)
    return cholesky_qr2(psi, sys.dV)


def kpoint_grid(sys: System, counts) -> tuple[np.ndarray, np.ndarray]:
    """Gamma-centred k-point grid: counts[a] points along each periodic axis (1 on
    Dirichlet axes), phases per cell theta_a = 2 pi j / counts[a], equal weights
    summing to 1.  Returns (theta (n_kpt, 3), weights (n_kpt,))."""
    for a in range(3):
        if sys.bc[a] == DIRICHLET and counts[a] != 1:
            raise ValueError("a Dirichlet axis takes a single k-point")
    grids = [2.0 * np.pi * np.arange(counts[a]) / counts[a] for a in range(3)]
    theta = np.array([[t1, t2, t3] for t3 in grids[2] for t2 in grids[1] for t1 in grids[0]])
    return theta, np.full(len(theta), 1.0 / len(theta))


def make_bloch_orbitals(sys: System, theta, n_orb: int | None = None, seed: int | None = None) -> np.ndarray:
    """Seeded complex Bloch orbitals, shape (n_kpt, N, n_orb) complex128: per k-point
    (u + i u') / sqrt(2) from two make_orbitals draws (periodic along periodic
    axes), times exp(i theta_a x_a / n_a) along each periodic axis (x_a the grid
    index), so that psi(x + n_a h_a) = exp(i theta_a) psi(x)."""
    theta = np.asarray(theta, dtype=np.float64).reshape(-1, 3)
    base = sys.seed if seed is None else seed
    n1, n2, n3 = sys.n
    idx = np.indices((n3, n2, n1))  # [x3, x2, x1]
    out = []
    for k, th in enumerate(theta):
        u = make_orbitals(sys, n_orb, base + 2 * k) + 1j * make_orbitals(sys, n_orb, base + 2 * k + 1)
        ph = np.zeros((n3, n2, n1))
        for a in range(3):
            if sys.bc[a] == PERIODIC:
                ph += th[a] * idx[2 - a] / sys.n[a]
        out.append(np.exp(1j * ph).reshape(-1, 1) * u / np.sqrt(2.0))
    return np.stack(out)


def random_field(n_total: int, n_rhs: int, seed: int) -> np.ndarray:
    """Plain N(0,1) right-hand sides, shape (n_total, n_rhs) float64."""
    return np.random.default_rng(seed).standard_normal((n_total, n_rhs))


def symmetric_pairs(n_orb: int):
    """Upper-triangular pair list (i <= j), row-major: the enumeration of the symmetric schedule."""
    return [(i, j) for i in range(n_orb) for j in range(i, n_orb)]


# ---------------------------------------------------------------------------
# The five workloads (Sec. 4 systems are replaced by synthetic stand-ins of the
# same grid sizes, spacings, boundary conditions and orbital counts).
# ---------------------------------------------------------------------------
def _cube(n):
    return (n, n, n)


C1 = System(n=_cube(32), h=(0.5,) * 3, bc=(DIRICHLET,) * 3, kernel=UNSCREENED, n_orb=4,
            n_centres=0, seed=1234, name="c1: 32^3 Dirichlet unscreened, 4 orbitals")
C2 = System(n=_cube(96), h=(0.25,) * 3, bc=(DIRICHLET,) * 3, kernel=UNSCREENED, n_orb=64,
            n_centres=24, seed=1235, name="c2: 96^3 Dirichlet unscreened, 64 orbitals")
_H3 = 23.47 / 80
C3 = System(n=_cube(80), h=(_H3,) * 3, bc=(PERIODIC,) * 3, kernel=SCREENED, n_orb=256,
            n_centres=192, seed=1236, name="c3: 80^3 periodic screened, 256 orbitals")

C4 = [
    System(n=_cube(40), h=(0.3,) * 3, bc=(DIRICHLET,) * 3, kernel=UNSCREENED, n_orb=16, n_centres=6, seed=1237,
           name="c4.0: 40^3 D unscreened, 16 orbitals"),
    System(n=(48, 48, 64), h=(0.3,) * 3, bc=(PERIODIC,) * 3, kernel=SCREENED, n_orb=32, n_centres=12, seed=1238,
           name="c4.1: 48x48x64 P screened, 32 orbitals"),
    System(n=_cube(56), h=(0.3,) * 3, bc=(DIRICHLET,) * 3, kernel=UNSCREENED, n_orb=48, n_centres=18, seed=1239,
           name="c4.2: 56^3 D unscreened, 48 orbitals"),
    System(n=(64, 64, 96), h=(0.3,) * 3, bc=(PERIODIC,) * 3, kernel=SCREENED, n_orb=64, n_centres=24, seed=1240,
           name="c4.3: 64x64x96 P screened, 64 orbitals"),
    System(n=_cube(72), h=(0.3,) * 3, bc=(DIRICHLET,) * 3, kernel=UNSCREENED, n_orb=80, n_centres=30, seed=1241,
           name="c4.4: 72^3 D unscreened, 80 orbitals"),
    System(n=_cube(80), h=(0.3,) * 3, bc=(PERIODIC,) * 3, kernel=SCREENED, n_orb=96, n_centres=36, seed=1242,
           name="c4.5: 80^3 P screened, 96 orbitals"),
    System(n=(48, 48, 120), h=(0.3,) * 3, bc=(PERIODIC, PERIODIC, DIRICHLET), kernel=UNSCREENED, n_orb=112,
           n_centres=42, seed=1243, name="c4.6: 48x48x120 slab (P,P,D) unscreened, 112 orbitals"),
    System(n=_cube(96), h=(0.3,) * 3, bc=(DIRICHLET,) * 3, kernel=SCREENED, n_orb=128, n_centres=48, seed=1244,
           name="c4.7: 96^3 D screened, 128 orbitals"),
]

C5 = C3  # differentiation workload runs on the 80^3 periodic screened system


# Bloch k-points: a slab periodic in x1 and x2 with vacuum (Dirichlet) along x3,
# unscreened kernel, 16 bands at each point of a 2 x 2 Gamma-centred k-grid.
K1 = System(n=(64, 64, 64), h=(0.3,) * 3, bc=(PERIODIC, PERIODIC, DIRICHLET), kernel=UNSCREENED, n_orb=16,
            n_centres=8, seed=61)
K1_KGRID = (2, 2, 1)


def n_pairs(n_orb: int, ordered: bool = False) -> int:
    return n_orb * n_orb if ordered else n_orb * (n_orb + 1) // 2


def useful_flops_per_pair(n) -> float:
    """Six mode products, 2 flops per multiply-add: 4 N (n1 + n2 + n3) (cost estimate of Sec. 3)."""
    N = n[0] * n[1] * n[2]
    return 4.0 * N * (n[0] + n[1] + n[2])
