"""FP64 CPU oracle for the exact-exchange apply through the Kronecker form of f(L).

TEST INFRASTRUCTURE ONLY.  This module is imported by the test suite, by the
package smoke check and by the CPU-baseline leg of the benchmark; the CUDA
library never calls it and shares no code with it.  It is written for a reader
checking it against the paper by eye: plain NumPy in float64, one step per line
of the method, no blocking, fusion or reordering.

Paper: "Efficient real space formalism for hybrid density functionals"
(arXiv 2406.16998).  Section / equation citations below refer to it.

Readings of places where the paper is silent or garbled (each also pinned by a
test in tests/test_oracle_pins.py):
  R1  Kronecker factor order.  With L = I3(x)I2(x)L1 + I3(x)L2(x)I1 + L3(x)I2(x)I1
      (Sec. 3, Eq. 11-12) and x1 the fastest grid index, the eigenvector matrix is
      V = V3(x)V2(x)V1; mode k of the grid array is contracted with Vk.
  R2  f(Lambda) is the diagonal with entries f(l1_i + l2_j + l3_k); the paper's
      sum-of-Kronecker expansion of f(Lambda) (Sec. 3) holds only for linear f.
  R3  Screened kernel: with mu = -lambda >= 0, f = (4 pi / mu)(1 - exp(-mu/(4 w^2))),
      f(0) = pi / w^2, i.e. the Fourier transform of erfc(w r)/r.  The paper's
      exponent -L/(16 pi w^2) (Sec. 2.2 and Sec. 3) does not reproduce that kernel.
  R4  w = 0.11 bohr^-1 (HSE06, the functional Sec. 4 names).
  R5  Unscreened f = -4 pi / lambda (Sec. 3).  Fully periodic + unscreened is
      singular (lambda = 0) and is rejected.
  R6  Centred 2m-order FD weights for d^2/dx^2 (order 12 <=> m = 6):
      w0 = -2 sum_{p=1}^m 1/p^2,  w_p = 2 (-1)^{p+1} (m!)^2 / (p^2 (m-p)! (m+p)!),
      all divided by h^2.
  R7  Dirichlet: n unknowns at x_i = (i+1) h, homogeneous zero values outside.
      Periodic: x_i = i h, circulant Lk.
  R8  Integrals become dV-weighted sums, dV = h1 h2 h3; occupations g default 1;
      real orbitals at the Gamma point, so conjugates drop (Sec. 2, Eq. 5 setting).
  R9  Pair enumeration: the symmetric (i <= j) and ordered schedules give the
      same VxPsi and E_x.
"""
from __future__ import annotations

import math
import numpy as np

DIRICHLET = 0
PERIODIC = 1
UNSCREENED = 0
SCREENED = 1


# ---------------------------------------------------------------------------
# 1D finite-difference Laplacians (Sec. 3, Eq. 12)
# ---------------------------------------------------------------------------
def fd_weights(order: int) -> np.ndarray:
    """Centred weights w_0..w_m (h = 1) of the order-2m second-derivative stencil (reading R6)."""
    if order < 2 or order % 2:
        raise ValueError("FD order must be even and >= 2")
    m = order // 2
    w = np.zeros(m + 1)
    w[0] = -2.0 * sum(1.0 / (p * p) for p in range(1, m + 1))
    fm = math.factorial(m)
    for p in range(1, m + 1):
        w[p] = 2.0 * (-1) ** (p + 1) * fm * fm / (p * p * math.factorial(m - p) * math.factorial(m + p))
    return w


def lap1d(n: int, h: float, bc: int, order: int) -> np.ndarray:
    """Dense n x n matrix Lk of d^2/dx^2 with the boundary condition built in (Sec. 3; R7)."""
    w = fd_weights(order) / (h * h)
    m = order // 2
    L = np.zeros((n, n))
    for i in range(n):
        for p in range(-m, m + 1):
            c = w[abs(p)]
            j = i + p
            if bc == PERIODIC:
                L[i, j % n] += c
            elif 0 <= j < n:
                L[i, j] += c
    return L


def eig1d(L: np.ndarray):
    """Eigendecomposition Lk Vk = Vk Lambda_k of the symmetric 1D matrix (Sec. 3, Eq. 13)."""
    lam, V = np.linalg.eigh(L)
    return lam, V


# ---------------------------------------------------------------------------
# Kernel f (Sec. 3, after Eq. 18; R3-R5)
# ---------------------------------------------------------------------------
def kernel_f(lam: np.ndarray, kind: int, omega: float = 0.11) -> np.ndarray:
    """f evaluated on eigenvalues lam of L (lam <= 0)."""
    mu = -np.asarray(lam, dtype=np.float64)
    if kind == UNSCREENED:
        if np.any(mu <= 0.0):
            raise ValueError("unscreened kernel is singular: L has a zero eigenvalue")
        return 4.0 * math.pi / mu
    if kind == SCREENED:
        out = np.empty_like(mu)
        z = mu == 0.0
        out[z] = math.pi / (omega * omega)
        nz = ~z
        out[nz] = -4.0 * math.pi * np.expm1(-mu[nz] / (4.0 * omega * omega)) / mu[nz]
        return out
    raise ValueError("unknown kernel kind")


class Plan:
    """Per-system setup: the three 1D eigendecompositions and the f(Lambda) table."""

    def __init__(self, n, h, bc, kind, omega=0.11, fd_order=12):
        self.n = tuple(int(x) for x in n)
        self.h = tuple(float(x) for x in h)
        self.bc = tuple(int(x) for x in bc)
        self.kind = int(kind)
        self.omega = float(omega)
        self.fd_order = int(fd_order)
        if self.kind == UNSCREENED and all(b == PERIODIC for b in self.bc):
            raise ValueError("unscreened kernel with periodic boundaries on all axes is singular")
        self.L = [lap1d(self.n[a], self.h[a], self.bc[a], self.fd_order) for a in range(3)]
        eig = [eig1d(Lk) for Lk in self.L]
        self.lam = [e[0] for e in eig]
        self.V = [e[1] for e in eig]
        # f(Lambda) diagonal, indexed like the grid: [k3, k2, k1]  (R2)
        lsum = (self.lam[2][:, None, None] + self.lam[1][None, :, None] + self.lam[0][None, None, :])
        self.fdiag = kernel_f(lsum, self.kind, self.omega)

    @property
    def N(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def dV(self):
        return self.h[0] * self.h[1] * self.h[2]


# ---------------------------------------------------------------------------
# X = f(L) B through Roth's relationship (Sec. 3, Eq. 19a,b)
# ---------------------------------------------------------------------------
def _as_cube(plan: Plan, b: np.ndarray) -> np.ndarray:
    n1, n2, n3 = plan.n
    return np.asarray(b, dtype=np.float64).reshape(n3, n2, n1)  # [x3, x2, x1]


def forward_transform(plan: Plan, b: np.ndarray) -> np.ndarray:
    """Spectral coefficients of one grid vector: slices V1^T B_k V2, then mode 3 with V3 (Eq. 19b)."""
    V1, V2, V3 = plan.V
    cube = _as_cube(plan, b)
    n1, n2, n3 = plan.n
    cols = np.empty((n1 * n2, n3))
    for k in range(n3):
        Bk = cube[k].T                      # frontal slice B(:, :, k), n1 x n2 (rows x1)
        Yk = V1.T @ Bk @ V2                 # modes 1 and 2
        cols[:, k] = Yk.reshape(-1, order="F")  # vec along n2 (x1 fastest)
    Y = cols @ V3                           # mode 3: (n1 n2) x n3 times V3
    return Y                                # [k1 + n1 k2, k3]


def inverse_transform(plan: Plan, Xt: np.ndarray) -> np.ndarray:
    """Grid values from spectral coefficients: slices V1 X_k V2^T, then mode 3 with V3^T (Eq. 19a)."""
    V1, V2, V3 = plan.V
    n1, n2, n3 = plan.n
    cols = np.empty((n1 * n2, n3))
    for k in range(n3):
        Xk = Xt[:, k].reshape(n1, n2, order="F")
        cols[:, k] = (V1 @ Xk @ V2.T).reshape(-1, order="F")
    X = cols @ V3.T
    return X.reshape(-1, order="F")          # x1 fastest, then x2, then x3


def fdiag_matrix(plan: Plan) -> np.ndarray:
    """f(Lambda) in the same [k1 + n1 k2, k3] layout as forward_transform's output."""
    n1, n2, n3 = plan.n
    return plan.fdiag.reshape(n3, n1 * n2).T


def apply_fL(plan: Plan, b: np.ndarray) -> np.ndarray:
    """X = f(L) b for one grid vector or a block of columns (N,) / (N, r)."""
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 2:
        return np.stack([apply_fL(plan, b[:, c]) for c in range(b.shape[1])], axis=1)
    Y = forward_transform(plan, b)
    Xt = fdiag_matrix(plan) * Y              # Hadamard scaling by f(Lambda)
    return inverse_transform(plan, Xt)


def dense_L(plan: Plan) -> np.ndarray:
    """Brute-force N x N Laplacian I3(x)I2(x)L1 + I3(x)L2(x)I1 + L3(x)I2(x)I1 (Sec. 3, Eq. 11)."""
    L1, L2, L3 = plan.L
    I1, I2, I3 = (np.eye(k) for k in plan.n)
    return np.kron(I3, np.kron(I2, L1)) + np.kron(I3, np.kron(L2, I1)) + np.kron(L3, np.kron(I2, I1))


def dense_fL(plan: Plan) -> np.ndarray:
    """Brute-force f(L) = V f(Lambda) V^T from a full eigendecomposition of the N x N matrix (Eq. 15)."""
    lam, V = np.linalg.eigh(dense_L(plan))
    return (V * kernel_f(lam, plan.kind, plan.omega)) @ V.T


# ---------------------------------------------------------------------------
# Exact exchange (Sec. 2, Eqs. 3-5 and 8-10, Gamma point, one spin channel)
# ---------------------------------------------------------------------------
def pair_list(n_orb: int, ordered: bool):
    if ordered:
        return [(i, j) for i in range(n_orb) for j in range(n_orb)]
    return [(i, j) for i in range(n_orb) for j in range(i, n_orb)]


def vx_apply(plan: Plan, psi: np.ndarray, occ=None, ordered: bool = False, pairs=None):
    """(Vx Psi)_i = -sum_j g_j psi_j * phi_ij with phi_ij = f(L)(psi_i * psi_j), and
    E_x = -1/2 dV sum_{i,j} g_i g_j <psi_i psi_j, phi_ij>.

    Returns (vx_psi (N, n_orb), e_x).  `pairs` restricts the sum to a sub-list of
    the chosen enumeration (used for sharded partial sums).
    """
    psi = np.asarray(psi, dtype=np.float64)
    n_orb = psi.shape[1]
    g = np.ones(n_orb) if occ is None else np.asarray(occ, dtype=np.float64)
    out = np.zeros_like(psi)
    e = 0.0
    if pairs is None:
        pairs = pair_list(n_orb, ordered)
    for (i, j) in pairs:
        rho = psi[:, i] * psi[:, j]
        phi = apply_fL(plan, rho)
        if ordered:
            out[:, i] -= g[j] * psi[:, j] * phi
            e += -0.5 * plan.dV * g[i] * g[j] * np.dot(rho, phi)
        else:
            out[:, i] -= g[j] * psi[:, j] * phi
            mult = 1.0
            if i != j:
                out[:, j] -= g[i] * psi[:, i] * phi
                mult = 2.0
            e += -0.5 * plan.dV * mult * g[i] * g[j] * np.dot(rho, phi)
    return out, e


def exchange_energy(plan: Plan, psi: np.ndarray, occ=None) -> float:
    """E_x alone via Parseval: sum over pairs of f(Lambda) * (V^T rho_ij)^2 (V orthogonal)."""
    psi = np.asarray(psi, dtype=np.float64)
    n_orb = psi.shape[1]
    g = np.ones(n_orb) if occ is None else np.asarray(occ, dtype=np.float64)
    F = fdiag_matrix(plan)
    e = 0.0
    for (i, j) in pair_list(n_orb, ordered=False):
        Y = forward_transform(plan, psi[:, i] * psi[:, j])
        mult = 1.0 if i == j else 2.0
        e += -0.5 * plan.dV * mult * g[i] * g[j] * float(np.sum(F * Y * Y))
    return e


def energy_gradient(plan: Plan, psi: np.ndarray, occ=None) -> np.ndarray:
    """dE_x / dpsi_k(r) = 2 dV g_k (Vx Psi)_k(r) for the discrete E_x above."""
    n_orb = psi.shape[1]
    g = np.ones(n_orb) if occ is None else np.asarray(occ, dtype=np.float64)
    vx, _ = vx_apply(plan, psi, occ)
    return 2.0 * plan.dV * vx * g[None, :]


# ---------------------------------------------------------------------------
# ACE tail (adaptively compressed exchange, cited in Sec. 4)
# ---------------------------------------------------------------------------
def ace(plan: Plan, psi: np.ndarray, vx_psi: np.ndarray):
    """W = Vx Psi;  M = dV Psi^T W;  -M = R^T R (Cholesky);  xi = W R^{-1}.

    Returns (xi, M, R).  The compressed operator -xi (dV xi^T .) reproduces W on Psi.
    """
    W = np.asarray(vx_psi, dtype=np.float64)
    M = plan.dV * (psi.T @ W)
    R = np.linalg.cholesky(-M).T            # upper triangular, R^T R = -M
    xi = np.linalg.solve(R.T, W.T).T        # xi = W R^{-1}
    return xi, M, R


def ace_apply(plan: Plan, xi: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """The compressed exchange operator applied to vectors: V_ACE phi = -xi (dV xi^T phi).

    xi: N x n_xi (from ace), phi: N x n_vec; returns N x n_vec.  On the occupied
    orbitals V_ACE Psi equals Vx Psi, which is what lets an SCF loop use V_ACE
    in place of Vx between rebuilds (the ACE construction Sec. 4 cites).
    """
    P = plan.dV * (xi.T @ phi)              # projections of phi on xi (dV inner product)
    return -(xi @ P)
