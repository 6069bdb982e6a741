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
  R10-R12 (multipole boundary values for isolated systems): see the section
      above apply_fL_multipole.
  R13-R16 (Bloch-periodic boundary conditions and k-point sums): see the section
      above lap1d_bloch.
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


def vx_apply(plan: Plan, psi: np.ndarray, occ=None, ordered: bool = False, pairs=None, l_max=None):
    """(Vx Psi)_i = -sum_j g_j psi_j * phi_ij with phi_ij = f(L)(psi_i * psi_j), and
    E_x = -1/2 dV sum_{i,j} g_i g_j <psi_i psi_j, phi_ij>.

    Returns (vx_psi (N, n_orb), e_x).  `pairs` restricts the sum to a sub-list of
    the chosen enumeration (used for sharded partial sums).  With l_max, each
    phi_ij takes the Dirichlet values of the multipole expansion of rho_ij up
    to order l_max (apply_fL_multipole) instead of zero boundary values.
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
        phi = apply_fL(plan, rho) if l_max is None else apply_fL_multipole(plan, rho, l_max)
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
# Dirichlet values from the multipole expansion of the source (Sec. 4: for
# isolated systems the boundary values of each linear system come from the
# multipole expansion of the Coulomb kernel and enter through the right-hand
# side).  Readings (R10-R12):
#  R10 The expansion is about the box centre c, c_a = (n_a + 1) h_a / 2, up to
#      order l_max (the paper gives no order); it applies to all-Dirichlet
#      boxes with the unscreened kernel (-del^2 phi = 4 pi rho).
#  R11 The exterior points are those the order-2m stencil of an interior point
#      reaches across one face: index -m..-1 or n_a..n_a+m-1 along one axis a,
#      interior along the other two, at x = (i + 1) h like the interior.
#  R12 Moving the known exterior values to the right-hand side of
#      L_full phi = -4 pi rho gives L phi = -4 pi (rho + L_ext phi_ext / (4 pi)),
#      i.e. phi = f(L) (rho + L_ext phi_ext / (4 pi)) with f = -4 pi / lambda.
# ---------------------------------------------------------------------------
def _require_isolated(plan: Plan):
    if plan.kind != UNSCREENED or any(b != DIRICHLET for b in plan.bc):
        raise ValueError("multipole boundary values need an all-Dirichlet box and the unscreened kernel")


def expansion_centre(plan: Plan) -> np.ndarray:
    return np.array([(plan.n[a] + 1) * plan.h[a] / 2.0 for a in range(3)])


def interior_points(plan: Plan) -> np.ndarray:
    """(N, 3) coordinates of the grid points, x1 fastest (R7)."""
    ax = [(np.arange(plan.n[a]) + 1) * plan.h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def exterior_points(plan: Plan):
    """Exterior points of R11 as a list of (axis, index along that axis, (M, 3)
    coordinates, (M,) flat index of the interior point sharing the other two
    indices); each face layer is one entry."""
    _require_isolated(plan)
    m = plan.fd_order // 2
    n1, n2, n3 = plan.n
    out = []
    for a in range(3):
        for i_a in list(range(-m, 0)) + list(range(plan.n[a], plan.n[a] + m)):
            idx = [np.arange(n1), np.arange(n2), np.arange(n3)]
            idx[a] = np.array([i_a])
            k3, k2, k1 = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
            k1, k2, k3 = k1.ravel(), k2.ravel(), k3.ravel()
            pts = np.stack([(k1 + 1) * plan.h[0], (k2 + 1) * plan.h[1], (k3 + 1) * plan.h[2]], axis=1)
            # the interior point on the same line along axis a, with index 0 (i_a < 0) or n_a - 1
            kk = [k1, k2, k3]
            kk[a] = np.full_like(kk[a], 0 if i_a < 0 else plan.n[a] - 1)
            flat = kk[0] + n1 * (kk[1] + n2 * kk[2])
            out.append((a, i_a, pts, flat))
    return out


def _spherical(v: np.ndarray):
    r = np.linalg.norm(v, axis=1)
    cos_t = np.where(r > 0, v[:, 2] / np.where(r > 0, r, 1.0), 1.0)
    phi = np.arctan2(v[:, 1], v[:, 0])
    return r, np.clip(cos_t, -1.0, 1.0), phi


def multipole_moments(plan: Plan, rho: np.ndarray, l_max: int):
    """Moments q[(l, m, t)] = dV sum_r rho(r) |r-c|^l P_l^m(cos theta) trig_t(m phi),
    t = 0 for cos and 1 for sin (m >= 1), about the expansion centre (R10)."""
    from scipy.special import lpmv
    r, ct, ph = _spherical(interior_points(plan) - expansion_centre(plan))
    q = {}
    for l in range(l_max + 1):
        for m in range(l + 1):
            base = plan.dV * rho * r ** l * lpmv(m, l, ct)
            q[(l, m, 0)] = float(np.sum(base * np.cos(m * ph)))
            if m > 0:
                q[(l, m, 1)] = float(np.sum(base * np.sin(m * ph)))
    return q


def multipole_potential(plan: Plan, q: dict, l_max: int, pts: np.ndarray) -> np.ndarray:
    """Potential of the moments at points outside the source (addition theorem of
    1/|p - r| in Legendre functions: sum_l r^l / p^(l+1) P_l(cos gamma) with
    P_l(cos gamma) = sum_m (2 - delta_m0) (l-m)!/(l+m)! P_l^m P_l^m cos(m (phi_p - phi_r)))."""
    from scipy.special import lpmv
    r, ct, ph = _spherical(pts - expansion_centre(plan))
    out = np.zeros(len(pts))
    for l in range(l_max + 1):
        for m in range(l + 1):
            w = (1.0 if m == 0 else 2.0) * math.factorial(l - m) / math.factorial(l + m)
            ang = q[(l, m, 0)] * np.cos(m * ph) + (q[(l, m, 1)] * np.sin(m * ph) if m > 0 else 0.0)
            out += w * lpmv(m, l, ct) * ang / r ** (l + 1)
    return out


def rhs_multipole(plan: Plan, rho: np.ndarray, l_max: int) -> np.ndarray:
    """rho + L_ext phi_ext / (4 pi) (R12): each exterior value reaches the interior
    points within m along its axis with the stencil weight of that distance."""
    _require_isolated(plan)
    rho = np.asarray(rho, dtype=np.float64)
    w = fd_weights(plan.fd_order)
    q = multipole_moments(plan, rho, l_max)
    b = rho.copy()
    n1, n2, n3 = plan.n
    stride = [1, n1, n1 * n2]
    m = plan.fd_order // 2
    for a, i_a, pts, flat in exterior_points(plan):
        vals = multipole_potential(plan, q, l_max, pts)
        # interior points i with |i - i_a| <= m along axis a
        lo, hi = (0, i_a + m) if i_a < 0 else (i_a - m, plan.n[a] - 1)
        edge = 0 if i_a < 0 else plan.n[a] - 1
        for i in range(max(lo, 0), min(hi, plan.n[a] - 1) + 1):
            d = abs(i - i_a)
            b[flat + (i - edge) * stride[a]] += w[d] / plan.h[a] ** 2 * vals / (4.0 * math.pi)
    return b


def apply_fL_multipole(plan: Plan, rho: np.ndarray, l_max: int) -> np.ndarray:
    """phi = f(L) (rho + L_ext phi_ext / (4 pi)): the solution of -del^2 phi = 4 pi rho
    whose values outside the box are the multipole expansion of rho's potential."""
    return apply_fL(plan, rhs_multipole(plan, rho, l_max))


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


# ---------------------------------------------------------------------------
# Bloch-periodic boundary conditions and k-point sums (Sec. 2.1, Eqs. 6-9: the
# orbitals are complex, the pair densities conj(psi_mq) phi_nk obey Bloch
# conditions at k - q along the extended axes, and the sums carry Brillouin-zone
# weights; Sec. 3: the 1D matrices may then be complex and wavevector
# dependent, and Eq. 19 contracts with the conjugated eigenvectors).  Readings:
#  R13 A k-point is given by its phase per cell along each periodic axis,
#      theta_a = k_a n_a h_a (radians); Dirichlet axes ignore it.  The Poisson
#      problem of the pair (mq, nk) takes the phases theta_k - theta_q.
#  R14 Bloch 1D matrix: a stencil point j = i + p that leaves the cell w times
#      (w = floor(j / n)) lands on j - w n with the factor exp(i w theta); the
#      matrix is Hermitian and theta = 0 gives the periodic one.
#  R15 The forward transform contracts each mode with conj(Vk) (the V^{*T} B V^{*}
#      of Eq. 19b), the inverse transform with Vk (Eq. 19a).
#  R16 Vx phi_nk = -sum_q w_q sum_m g_mq psi_mq f(L_{k-q})(conj(psi_mq) phi_nk) and
#      E_x = -1/2 dV sum_k w_k sum_n g_nk sum_q w_q sum_m g_mq <rho, f rho> with
#      rho = conj(psi_mq) psi_nk and <a, b> = sum_r conj(a) b (Eqs. 7-8), for one
#      spin channel; the spin sum of Eq. 6 adds independent channels.
# ---------------------------------------------------------------------------
def lap1d_bloch(n: int, h: float, order: int, theta: float) -> np.ndarray:
    """Dense complex n x n matrix of d^2/dx^2 with the Bloch condition u(x + n h) = e^{i theta} u(x) (R14)."""
    w = fd_weights(order) / (h * h)
    m = order // 2
    L = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        for p in range(-m, m + 1):
            j = i + p
            wraps = j // n                  # floor division: cells crossed, with sign
            L[i, j - wraps * n] += w[abs(p)] * np.exp(1j * wraps * theta)
    return L


class BlochPlan(Plan):
    """The set-up of a Plan for the Poisson problems at one phase difference theta
    (3 values, radians per cell; ignored on Dirichlet axes): complex eigenvectors
    along the periodic axes (R13-R14), real ones along the Dirichlet axes."""

    def __init__(self, base: Plan, theta):
        self.n, self.h, self.bc = base.n, base.h, base.bc
        self.kind, self.omega, self.fd_order = base.kind, base.omega, base.fd_order
        self.theta = tuple(float(t) for t in theta)
        self.L = []
        for a in range(3):
            if self.bc[a] == PERIODIC:
                self.L.append(lap1d_bloch(self.n[a], self.h[a], self.fd_order, self.theta[a]))
            else:
                self.L.append(lap1d(self.n[a], self.h[a], self.bc[a], self.fd_order).astype(np.complex128))
        eig = [np.linalg.eigh(Lk) for Lk in self.L]
        self.lam = [e[0] for e in eig]
        self.V = [e[1] for e in eig]
        lsum = (self.lam[2][:, None, None] + self.lam[1][None, :, None] + self.lam[0][None, None, :])
        self.fdiag = kernel_f(lsum, self.kind, self.omega)


def forward_transform_bloch(plan: BlochPlan, b: np.ndarray) -> np.ndarray:
    """Spectral coefficients: slices V1^H B_k conj(V2), then mode 3 with conj(V3) (Eq. 19b, R15)."""
    V1, V2, V3 = plan.V
    n1, n2, n3 = plan.n
    cube = np.asarray(b, dtype=np.complex128).reshape(n3, n2, n1)
    cols = np.empty((n1 * n2, n3), dtype=np.complex128)
    for k in range(n3):
        Bk = cube[k].T
        Yk = V1.conj().T @ Bk @ V2.conj()
        cols[:, k] = Yk.reshape(-1, order="F")
    return cols @ V3.conj()


def inverse_transform_bloch(plan: BlochPlan, Xt: np.ndarray) -> np.ndarray:
    """Grid values: slices V1 X_k V2^T, then mode 3 with V3^T (Eq. 19a)."""
    V1, V2, V3 = plan.V
    n1, n2, n3 = plan.n
    cols = np.empty((n1 * n2, n3), dtype=np.complex128)
    for k in range(n3):
        Xk = Xt[:, k].reshape(n1, n2, order="F")
        cols[:, k] = (V1 @ Xk @ V2.T).reshape(-1, order="F")
    return (cols @ V3.T).reshape(-1, order="F")


def apply_fL_bloch(plan: BlochPlan, b: np.ndarray) -> np.ndarray:
    """X = f(L_theta) b for one complex grid vector (N,) (Sec. 3, Eq. 19 with complex Vk)."""
    Y = forward_transform_bloch(plan, b)
    return inverse_transform_bloch(plan, fdiag_matrix(plan) * Y)


def _kpoint_args(theta, wk, psi, occ):
    theta = np.asarray(theta, dtype=np.float64).reshape(-1, 3)
    wk = np.asarray(wk, dtype=np.float64).reshape(-1)
    psi = np.asarray(psi, dtype=np.complex128)      # (n_kpt, N, n_orb)
    n_kpt, _, n_orb = psi.shape
    if theta.shape[0] != n_kpt or wk.shape[0] != n_kpt:
        raise ValueError("theta, weights and orbitals disagree on the number of k-points")
    g = np.ones((n_kpt, n_orb)) if occ is None else np.asarray(occ, dtype=np.float64).reshape(n_kpt, n_orb)
    return theta, wk, psi, g


def vx_apply_kpoint(base: Plan, theta, wk, psi, occ, k: int, phi: np.ndarray) -> np.ndarray:
    """Vx applied to vectors phi (N, n_vec) at k-point k (R16): for every q and band m,
    phi_v -> -w_q g_mq psi_mq f(L_{theta_k - theta_q})(conj(psi_mq) phi_v), summed."""
    theta, wk, psi, g = _kpoint_args(theta, wk, psi, occ)
    phi = np.asarray(phi, dtype=np.complex128)
    out = np.zeros_like(phi)
    for q in range(psi.shape[0]):
        plan = BlochPlan(base, theta[k] - theta[q])
        for m in range(psi.shape[2]):
            for v in range(phi.shape[1]):
                rho = np.conj(psi[q][:, m]) * phi[:, v]
                out[:, v] -= wk[q] * g[q, m] * psi[q][:, m] * apply_fL_bloch(plan, rho)
    return out


def vx_kpoints(base: Plan, theta, wk, psi, occ=None):
    """Vx psi_nk at every k-point (n_kpt, N, n_orb) and E_x = 1/2 dV sum_k w_k sum_n
    g_nk <psi_nk, Vx psi_nk> (the same sum as Eq. 8 after the Poisson solve, R16)."""
    theta, wk, psi, g = _kpoint_args(theta, wk, psi, occ)
    vx = np.stack([vx_apply_kpoint(base, theta, wk, psi, g, k, psi[k]) for k in range(psi.shape[0])])
    e = 0.0
    for k in range(psi.shape[0]):
        for n in range(psi.shape[2]):
            e += 0.5 * base.dV * wk[k] * g[k, n] * np.vdot(psi[k][:, n], vx[k][:, n]).real
    return vx, e


def exchange_energy_kpoints(base: Plan, theta, wk, psi, occ=None) -> float:
    """E_x of Eq. 8 through Parseval: -1/2 dV sum w_k w_q g_nk g_mq sum f(Lambda) |V^H rho|^2."""
    theta, wk, psi, g = _kpoint_args(theta, wk, psi, occ)
    e = 0.0
    for k in range(psi.shape[0]):
        for q in range(psi.shape[0]):
            plan = BlochPlan(base, theta[k] - theta[q])
            F = fdiag_matrix(plan)
            for n in range(psi.shape[2]):
                for m in range(psi.shape[2]):
                    Y = forward_transform_bloch(plan, np.conj(psi[q][:, m]) * psi[k][:, n])
                    e += -0.5 * base.dV * wk[k] * wk[q] * g[k, n] * g[q, m] * float(np.sum(F * np.abs(Y) ** 2))
    return e
