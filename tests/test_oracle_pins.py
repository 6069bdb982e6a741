"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No test here compares the oracle with itself: each checks a closed form, an
identity the paper states (Sec. 3, Eqs. 11-19), an independent derivation, a
brute-force dense computation, or a continuum limit.  All run on the CPU.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import erf

import oracle
from oracle import DIRICHLET as D, PERIODIC as P, UNSCREENED as U, SCREENED as S
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def exact_weights(order):
    """Independent derivation: solve the Vandermonde moment system in exact rationals.

    Symmetric stencil sum_{p=-m}^{m} c_p f(p) = f''(0) for f = x^{2q}, q = 0..m.
    """
    m = order // 2
    # unknowns c_0, c_1..c_m (c_{-p} = c_p); equations for x^0, x^2, ..., x^{2m}
    A = [[Fraction(0)] * (m + 1) for _ in range(m + 1)]
    rhs = [Fraction(0)] * (m + 1)
    for q in range(m + 1):
        A[q][0] = Fraction(1 if q == 0 else 0)
        for p in range(1, m + 1):
            A[q][p] = Fraction(2 * p ** (2 * q))
        rhs[q] = Fraction(2 if q == 1 else 0)
    # Gauss-Jordan in rationals
    n = m + 1
    M = [row[:] + [rhs[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def stencil_matrix(n, h, bc, order):
    """Sparse 1D second-derivative stencil built from the exact rational weights."""
    w = [float(x) for x in exact_weights(order)]
    m = order // 2
    rows, cols, vals = [], [], []
    for i in range(n):
        for p in range(-m, m + 1):
            j = i + p
            if bc == P:
                j %= n
            elif not (0 <= j < n):
                continue
            rows.append(i)
            cols.append(j)
            vals.append(w[abs(p)] / h ** 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def sparse_laplacian(plan):
    L1, L2, L3 = (stencil_matrix(plan.n[a], plan.h[a], plan.bc[a], plan.fd_order) for a in range(3))
    I1, I2, I3 = (sp.identity(k, format="csr") for k in plan.n)
    return (sp.kron(I3, sp.kron(I2, L1)) + sp.kron(I3, sp.kron(L2, I1)) + sp.kron(L3, sp.kron(I2, I1))).tocsr()


def small_orbitals(n, h, bc, n_orb, seed, kernel=U):
    sysd = workloads.System(n=n, h=h, bc=bc, kernel=kernel, n_orb=n_orb, n_centres=3, seed=seed)
    return workloads.make_orbitals(sysd), sysd


# ---------------------------------------------------------------- P1: FD weights
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_fd_weights_match_exact_rational_derivation(order):
    w = oracle.fd_weights(order)
    ex = exact_weights(order)
    assert np.max(np.abs(w - np.array([float(x) for x in ex]))) < 1e-14


def test_fd_weights_match_textbook_table():
    with open(os.path.join(GOLDEN, "fd_weights_textbook.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            order, vals = line.split(":")
            ref = np.array([float(Fraction(v)) for v in vals.split()])
            assert np.max(np.abs(oracle.fd_weights(int(order)) - ref)) < 1e-15


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_fd_weights_exact_on_polynomials(order):
    m = order // 2
    w = oracle.fd_weights(order)
    x0 = 0.37
    for q in range(0, 2 * m + 2):
        f = lambda x: x ** q
        d2 = q * (q - 1) * x0 ** (q - 2) if q >= 2 else 0.0
        approx = w[0] * f(x0) + sum(w[p] * (f(x0 + p) + f(x0 - p)) for p in range(1, m + 1))
        assert abs(approx - d2) <= 1e-9 * max(1.0, abs(d2)) * (m + 1) ** q / 10


def test_fd_symbol_order12():
    w = oracle.fd_weights(12)
    th = np.linspace(1e-3, 0.9, 200)
    sym = w[0] + 2 * sum(w[p] * np.cos(p * th) for p in range(1, 7))
    # symbol = -theta^2 + O(theta^14): error within rounding plus a theta^14 term
    assert np.all(np.abs(sym + th ** 2) <= 1e-14 + 1e-3 * th ** 14)
    # and the theta^14 term is really there (order exactly 12, not higher)
    assert np.abs(sym[-1] + th[-1] ** 2) > 1e-6 * th[-1] ** 14
    th_all = np.linspace(0, np.pi, 2001)
    sym_all = w[0] + 2 * sum(w[p] * np.cos(p * th_all) for p in range(1, 7))
    assert sym_all.max() <= 1e-15 and abs(sym_all.min() + 7.0729) < 1e-3


# ---------------------------------------------------------------- P2/P3: 1D closed forms
@pytest.mark.parametrize("n,h", [(9, 0.5), (16, 0.3)])
def test_order2_dirichlet_closed_form(n, h):
    L = oracle.lap1d(n, h, D, 2)
    k = np.arange(1, n + 1)
    lam = -(4 / h ** 2) * np.sin(k * np.pi / (2 * (n + 1))) ** 2
    i = np.arange(1, n + 1)
    V = np.sqrt(2 / (n + 1)) * np.sin(np.outer(i, k) * np.pi / (n + 1))
    assert np.max(np.abs(L @ V - V * lam)) < 1e-12 / h ** 2
    lam_o, V_o = oracle.eig1d(L)
    assert np.max(np.abs(np.sort(lam) - lam_o)) < 1e-12 / h ** 2
    # eigenvectors agree up to sign (simple spectrum)
    Vs = V[:, np.argsort(lam)]
    assert np.max(np.abs(np.abs(np.sum(Vs * V_o, axis=0)) - 1)) < 1e-12


@pytest.mark.parametrize("n,order", [(8, 2), (12, 12), (15, 12), (7, 6)])
def test_periodic_closed_form(n, order):
    h = 0.41
    L = oracle.lap1d(n, h, P, order)
    w = [float(x) for x in exact_weights(order)]
    m = order // 2
    th = 2 * np.pi * np.arange(n) / n
    lam = (w[0] + 2 * sum(w[p] * np.cos(p * th) for p in range(1, m + 1))) / h ** 2
    x = np.arange(n)
    for kk in range(n):
        c = np.cos(th[kk] * x)
        s = np.sin(th[kk] * x)
        assert np.max(np.abs(L @ c - lam[kk] * c)) < 1e-11
        assert np.max(np.abs(L @ s - lam[kk] * s)) < 1e-11
    lam_o, V_o = oracle.eig1d(L)
    assert np.max(np.abs(np.sort(lam) - lam_o)) < 1e-11
    assert np.max(np.abs(V_o.T @ V_o - np.eye(n))) < 1e-13


def test_order12_dirichlet_needs_dense_eig():
    # for order > 2 the truncated Toeplitz matrix is not diagonalised by sines (Sec. 3 keeps a dense eig)
    n, h = 32, 0.5
    L = oracle.lap1d(n, h, D, 12)
    k = np.arange(1, n + 1)
    V = np.sqrt(2 / (n + 1)) * np.sin(np.outer(k, k) * np.pi / (n + 1))
    off = V.T @ L @ V
    assert np.max(np.abs(off - np.diag(np.diag(off)))) > 0.1
    lam, Vo = oracle.eig1d(L)
    assert np.max(np.abs(L @ Vo - Vo * lam)) < 1e-12 * np.abs(lam).max()
    assert lam.max() < 0


# ---------------------------------------------------------------- kernel f
def test_kernel_f_values():
    lam = np.array([-1.0, -0.25, -4.0])
    assert np.allclose(oracle.kernel_f(lam, U), 4 * np.pi / -lam, rtol=1e-15)
    w = 0.11
    ref = 4 * np.pi / -lam * (1 - np.exp(lam / (4 * w * w)))
    assert np.allclose(oracle.kernel_f(lam, S, w), ref, rtol=1e-13)
    assert oracle.kernel_f(np.array([0.0]), S, w)[0] == pytest.approx(np.pi / w ** 2, rel=1e-15)
    # continuity at mu -> 0
    assert oracle.kernel_f(np.array([-1e-10]), S, w)[0] == pytest.approx(np.pi / w ** 2, rel=1e-8)
    with pytest.raises(ValueError):
        oracle.kernel_f(np.array([0.0]), U)


def test_fully_periodic_unscreened_rejected():
    with pytest.raises(ValueError):
        oracle.Plan((6, 6, 6), (0.5,) * 3, (P, P, P), U)
    oracle.Plan((6, 6, 6), (0.5,) * 3, (P, P, D), U)  # slab is fine


# ---------------------------------------------------------------- P4: eigenvectors of L
def _closed_vec(n, h, bc, order, mode):
    if bc == D:
        assert order == 2
        i = np.arange(1, n + 1)
        v = np.sin(i * mode * np.pi / (n + 1))
        lam = -(4 / h ** 2) * np.sin(mode * np.pi / (2 * (n + 1))) ** 2
    else:
        w = [float(x) for x in exact_weights(order)]
        th = 2 * np.pi * mode / n
        v = np.cos(th * np.arange(n))
        lam = (w[0] + 2 * sum(w[p] * np.cos(p * th) for p in range(1, order // 2 + 1))) / h ** 2
    return v, lam


@pytest.mark.parametrize("n,h,bc,kind,order,modes", [
    ((7, 9, 11), (0.5, 0.45, 0.4), (D, P, D), U, 2, (2, 3, 5)),
    ((8, 10, 12), (0.4, 0.5, 0.3), (P, P, P), S, 12, (1, 3, 0)),
    ((10, 6, 9), (0.3, 0.3, 0.3), (P, D, P), S, 2, (4, 1, 2)),
])
def test_fL_on_kronecker_eigenvector(n, h, bc, kind, order, modes):
    plan = oracle.Plan(n, h, bc, kind, fd_order=order)
    vs, lams = zip(*[_closed_vec(n[a], h[a], bc[a], order, modes[a]) for a in range(3)])
    v = np.kron(vs[2], np.kron(vs[1], vs[0]))           # x1 fastest
    fl = oracle.kernel_f(np.array([sum(lams)]), kind)[0]
    x = oracle.apply_fL(plan, v)
    assert np.max(np.abs(x - fl * v)) < 1e-12 * fl * np.abs(v).max()


def test_screened_constant_mode_periodic():
    plan = oracle.Plan((8, 9, 10), (0.3, 0.3, 0.3), (P, P, P), S, omega=0.11)
    x = oracle.apply_fL(plan, np.ones(plan.N))
    assert np.max(np.abs(x - np.pi / 0.11 ** 2)) < 1e-10 * np.pi / 0.11 ** 2


# ---------------------------------------------------------------- P5 / P11: Poisson identity, CG
@pytest.mark.parametrize("n,h,bc", [((10, 11, 12), (0.5, 0.45, 0.4), (D, D, D)),
                                    ((8, 9, 14), (0.5, 0.5, 0.35), (P, P, D))])
def test_minus_L_fL_is_4pi(n, h, bc):
    plan = oracle.Plan(n, h, bc, U)
    L = sparse_laplacian(plan)
    b = workloads.random_field(plan.N, 1, 7)[:, 0]
    x = oracle.apply_fL(plan, b)
    r = -(L @ x) - 4 * np.pi * b
    assert np.max(np.abs(r)) < 1e-11 * 4 * np.pi * np.abs(b).max() * (np.abs(L).max())


def test_cg_cross_check_unscreened_dirichlet():
    plan = oracle.Plan((9, 10, 11), (0.5,) * 3, (D, D, D), U)
    A = -sparse_laplacian(plan)
    b = workloads.random_field(plan.N, 1, 3)[:, 0]
    x_cg, info = spla.cg(A, 4 * np.pi * b, rtol=1e-14, atol=0.0, maxiter=20000)
    assert info == 0
    x = oracle.apply_fL(plan, b)
    assert np.max(np.abs(x - x_cg)) < 1e-9 * np.abs(x).max()


# ---------------------------------------------------------------- P6: symmetry, positivity
@pytest.mark.parametrize("bc,kind", [((D, D, D), U), ((P, P, P), S), ((P, D, P), U)])
def test_fL_symmetric_positive(bc, kind):
    plan = oracle.Plan((7, 8, 9), (0.4, 0.5, 0.45), bc, kind)
    a, b = workloads.random_field(plan.N, 2, 11).T
    fa, fb = oracle.apply_fL(plan, a), oracle.apply_fL(plan, b)
    assert abs(a @ fb - fa @ b) < 1e-12 * abs(a @ fb) + 1e-12 * np.linalg.norm(a) * np.linalg.norm(fb)
    assert b @ fb > 0 and a @ fa > 0


# ---------------------------------------------------------------- P8: brute force dense
@pytest.mark.parametrize("n,h,bc,kind", [
    ((6, 7, 8), (0.5, 0.4, 0.3), (P, P, D), U),
    ((5, 6, 7), (0.6, 0.5, 0.4), (D, D, D), U),
    ((6, 5, 7), (0.5, 0.5, 0.5), (P, P, P), S),
    ((7, 6, 5), (0.4, 0.5, 0.6), (D, P, D), S),
])
def test_apply_fL_matches_dense_matrix_function(n, h, bc, kind):
    plan = oracle.Plan(n, h, bc, kind)
    G = oracle.dense_fL(plan)
    B = workloads.random_field(plan.N, 3, 5)
    X = oracle.apply_fL(plan, B)
    assert np.max(np.abs(G @ B - X)) < 1e-11 * np.abs(X).max()


def test_vx_and_energy_match_dense_definition():
    n, h, bc = (6, 7, 8), (0.5, 0.45, 0.4), (D, P, D)
    psi, sysd = small_orbitals(n, h, bc, 4, 21)
    plan = oracle.Plan(n, h, bc, U)
    G = oracle.dense_fL(plan)
    g = np.array([1.0, 0.7, 0.4, 1.0])
    vx_ref = np.zeros_like(psi)
    e_ref = 0.0
    for a in range(4):          # Eq. 3-4 written out with the dense Green's matrix
        for b in range(4):
            phi = G @ (psi[:, b] * psi[:, a])
            vx_ref[:, a] -= g[b] * psi[:, b] * phi
            e_ref -= 0.5 * g[a] * g[b] * plan.dV * np.sum(psi[:, a] * phi * psi[:, b])
    vx, e = oracle.vx_apply(plan, psi, g)
    assert np.max(np.abs(vx - vx_ref)) < 1e-12 * np.abs(vx_ref).max()
    assert abs(e - e_ref) < 1e-12 * abs(e_ref)


# ---------------------------------------------------------------- P7: Vx on the occupied space
def test_vx_projection_symmetric_nsd_and_trace():
    psi, sysd = small_orbitals((8, 9, 10), (0.45,) * 3, (D, D, D), 5, 31)
    plan = oracle.Plan(sysd.n, sysd.h, sysd.bc, U)
    vx, e = oracle.vx_apply(plan, psi)
    M = plan.dV * psi.T @ vx
    assert np.max(np.abs(M - M.T)) < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).max() < 1e-12 * np.abs(M).max()
    assert abs(e - 0.5 * np.trace(M)) < 1e-12 * abs(e)
    assert e < 0
    assert abs(oracle.exchange_energy(plan, psi) - e) < 1e-12 * abs(e)


def test_energy_parseval_with_occupations():
    psi, sysd = small_orbitals((7, 8, 9), (0.5,) * 3, (P, P, P), 4, 41, kernel=S)
    plan = oracle.Plan(sysd.n, sysd.h, sysd.bc, S)
    g = np.array([1.0, 0.5, 0.25, 0.9])
    vx, e = oracle.vx_apply(plan, psi, g)
    M = plan.dV * psi.T @ vx
    assert abs(e - 0.5 * np.sum(g * np.diag(M))) < 1e-12 * abs(e)
    assert abs(oracle.exchange_energy(plan, psi, g) - e) < 1e-12 * abs(e)


# ---------------------------------------------------------------- P9: invariances
def test_invariances():
    n, h, bc = (6, 7, 9), (0.5, 0.45, 0.4), (D, P, D)
    psi, sysd = small_orbitals(n, h, bc, 3, 51, kernel=S)
    plan = oracle.Plan(n, h, bc, S)
    vx, e = oracle.vx_apply(plan, psi)
    # ordered and symmetric enumerations agree
    vx_o, e_o = oracle.vx_apply(plan, psi, ordered=True)
    assert np.max(np.abs(vx - vx_o)) < 1e-12 * np.abs(vx).max() and abs(e - e_o) < 1e-12 * abs(e)
    # orbital rotation: E invariant, VxPsi -> VxPsi U
    U_, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((3, 3)))
    vx_r, e_r = oracle.vx_apply(plan, psi @ U_)
    assert abs(e_r - e) < 1e-12 * abs(e)
    assert np.max(np.abs(vx_r - vx @ U_)) < 1e-12 * np.abs(vx).max()
    # scaling: Vx(c psi) = c^3 Vx(psi), E(c psi) = c^4 E(psi)
    c = 1.7
    vx_c, e_c = oracle.vx_apply(plan, c * psi)
    assert np.max(np.abs(vx_c - c ** 3 * vx)) < 1e-12 * np.abs(vx_c).max()
    assert abs(e_c - c ** 4 * e) < 1e-12 * abs(e_c)
    # axis permutation: swap x1 <-> x3
    n1, n2, n3 = n
    cube = psi.reshape(n3, n2, n1, 3)
    psi_p = np.ascontiguousarray(cube.transpose(2, 1, 0, 3)).reshape(-1, 3)
    plan_p = oracle.Plan((n3, n2, n1), (h[2], h[1], h[0]), (bc[2], bc[1], bc[0]), S)
    vx_p, e_p = oracle.vx_apply(plan_p, psi_p)
    vx_back = vx_p.reshape(n1, n2, n3, 3).transpose(2, 1, 0, 3).reshape(-1, 3)
    assert abs(e_p - e) < 1e-12 * abs(e)
    assert np.max(np.abs(vx_back - vx)) < 1e-12 * np.abs(vx).max()


def test_degenerate_cases():
    plan = oracle.Plan((5, 6, 7), (0.5,) * 3, (D, D, D), U)
    # zero orbital contributes nothing
    psi = np.zeros((plan.N, 2))
    psi[:, 0] = workloads.random_field(plan.N, 1, 2)[:, 0]
    vx, e = oracle.vx_apply(plan, psi)
    assert np.all(vx[:, 1] == 0)
    vx1, e1 = oracle.vx_apply(plan, psi[:, :1])
    assert np.max(np.abs(vx1[:, 0] - vx[:, 0])) == 0 and e1 == e
    # a single orbital: Vx psi = -psi f(L)(psi^2), E = -1/2 dV <psi^2, f(L) psi^2>
    p = psi[:, 0]
    phi = oracle.apply_fL(plan, p * p)
    assert np.max(np.abs(vx1[:, 0] + p * phi)) < 1e-13 * np.abs(p * phi).max()


# ---------------------------------------------------------------- P10: continuum limit (constants 4 pi, w)
def test_screened_periodic_gaussian_continuum_limit():
    Lbox, n = 12.0, 60
    h = Lbox / n
    w, alpha = 0.11, 1.5
    plan = oracle.Plan((n, n, n), (h,) * 3, (P, P, P), S, omega=w)
    x = np.arange(n) * h
    c0 = np.array([5.9, 6.1, 6.05])

    def d(ax):
        dd = x - c0[ax]
        return (dd + Lbox / 2) % Lbox - Lbox / 2
    dx, dy, dz = d(0), d(1), d(2)
    r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
    rho = (alpha / np.pi) ** 1.5 * np.exp(-alpha * r2)
    phi = oracle.apply_fL(plan, rho.reshape(-1)).reshape(n, n, n)
    cc = 1.0 / np.sqrt(1.0 / alpha + 1.0 / w ** 2)
    rng = np.random.default_rng(1)
    pts = rng.integers(0, n, size=(40, 3))
    err = 0.0
    ref_max = 0.0
    for (i3, i2, i1) in pts:
        r0 = np.array([x[i1], x[i2], x[i3]])
        tot = 0.0
        for a in range(-4, 5):
            for b in range(-4, 5):
                for c in range(-4, 5):
                    rr = np.linalg.norm(r0 - c0 + Lbox * np.array([a, b, c]))
                    if rr < 1e-12:
                        tot += 2 * np.sqrt(alpha / np.pi) - 2 * cc / np.sqrt(np.pi)
                    else:
                        tot += (erf(np.sqrt(alpha) * rr) - erf(cc * rr)) / rr
        err = max(err, abs(phi[i3, i2, i1] - tot))
        ref_max = max(ref_max, abs(tot))
    assert err < 1e-5 * ref_max


# ---------------------------------------------------------------- P12: gradient
def test_energy_gradient_finite_differences():
    psi, sysd = small_orbitals((6, 7, 8), (0.5,) * 3, (D, D, D), 3, 61)
    plan = oracle.Plan(sysd.n, sysd.h, sysd.bc, U)
    g = np.array([1.0, 0.8, 0.6])
    grad = oracle.energy_gradient(plan, psi, g)
    rng = np.random.default_rng(5)
    step = 1e-4
    for _ in range(16):
        r, k = int(rng.integers(plan.N)), int(rng.integers(3))
        pp, pm = psi.copy(), psi.copy()
        pp[r, k] += step
        pm[r, k] -= step
        fd = (oracle.exchange_energy(plan, pp, g) - oracle.exchange_energy(plan, pm, g)) / (2 * step)
        assert abs(fd - grad[r, k]) < 1e-7 * np.abs(grad).max()


# ---------------------------------------------------------------- ACE tail
def test_ace_reproduces_vx_on_occupied_space():
    psi, sysd = small_orbitals((7, 8, 9), (0.45,) * 3, (P, P, D), 4, 71)
    plan = oracle.Plan(sysd.n, sysd.h, sysd.bc, U)
    vx, _ = oracle.vx_apply(plan, psi)
    xi, M, R = oracle.ace(plan, psi, vx)
    assert np.max(np.abs(np.tril(R, -1))) == 0.0
    assert np.max(np.abs(R.T @ R + M)) < 1e-12 * np.abs(M).max()
    Vace_psi = -xi @ (plan.dV * xi.T @ psi)
    assert np.max(np.abs(Vace_psi - vx)) < 1e-11 * np.abs(vx).max()


def test_ace_apply_is_vx_on_occupied_space_and_projector_elsewhere():
    """V_ACE = -xi (dV xi^T .) must give Vx Psi on the orbitals (checked against the
    pair-by-pair Vx apply, not against a retyped formula), be symmetric and
    negative semidefinite in the dV inner product, and vanish on every vector
    dV-orthogonal to span(Vx Psi)."""
    psi, sysd = small_orbitals((8, 7, 6), (0.5,) * 3, (D, P, D), 5, 73)
    plan = oracle.Plan(sysd.n, sysd.h, sysd.bc, S)
    vx, _ = oracle.vx_apply(plan, psi)
    xi, M, _ = oracle.ace(plan, psi, vx)
    assert np.max(np.abs(oracle.ace_apply(plan, xi, psi) - vx)) < 1e-11 * np.abs(vx).max()
    # on the occupied space V_ACE has the matrix elements of Vx
    Vp = oracle.ace_apply(plan, xi, psi)
    assert np.max(np.abs(plan.dV * psi.T @ Vp - M)) < 1e-11 * np.abs(M).max()
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal((plan.N, 3)), rng.standard_normal((plan.N, 3))
    Va, Vb = oracle.ace_apply(plan, xi, a), oracle.ace_apply(plan, xi, b)
    lhs, rhs = a.T @ Vb, Va.T @ b
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.abs(lhs).max()
    assert np.all(np.diag(b.T @ Vb) <= 0.0)
    # component of b orthogonal to span(vx): least-squares residual, independent of xi
    coef, *_ = np.linalg.lstsq(vx, b, rcond=None)
    b_perp = b - vx @ coef
    assert np.max(np.abs(oracle.ace_apply(plan, xi, b_perp))) < 1e-11 * np.abs(Vb).max()
    # rank: at most n_orb nonzero singular values
    sv = np.linalg.svd(oracle.ace_apply(plan, xi, rng.standard_normal((plan.N, 12))), compute_uv=False)
    assert np.all(sv[psi.shape[1]:] < 1e-11 * sv[0])


# ---------------------------------------------------------------- multipole boundary values
def _gaussian(plan, centre, alpha):
    """Normalised Gaussian charge (total charge 1) sampled on the grid."""
    d = oracle.interior_points(plan) - np.asarray(centre)
    return (alpha / math.pi) ** 1.5 * np.exp(-alpha * np.sum(d * d, axis=1))


def test_multipole_values_are_the_legendre_series_and_converge_to_coulomb():
    """Exterior values from the moments equal the Legendre series of 1/|p - r|
    summed over the source directly (the addition theorem, written here the
    other way round), and approach the direct Coulomb sum as l_max grows."""
    from scipy.special import eval_legendre
    plan = oracle.Plan((16, 14, 18), (0.6, 0.6, 0.6), (D, D, D), U)
    c = oracle.expansion_centre(plan)
    rho = _gaussian(plan, c + np.array([0.4, -0.3, 0.25]), 4.0)
    src = oracle.interior_points(plan) - c
    rs = np.linalg.norm(src, axis=1)
    pts = np.concatenate([e[2] for e in oracle.exterior_points(plan)])[::7]
    rel = pts - c
    rp = np.linalg.norm(rel, axis=1)
    coul = np.array([plan.dV * np.sum(rho / np.linalg.norm(p - oracle.interior_points(plan), axis=1)) for p in pts])
    errs = []
    for l_max in (0, 2, 4, 8):
        q = oracle.multipole_moments(plan, rho, l_max)
        vals = oracle.multipole_potential(plan, q, l_max, pts)
        series = np.zeros(len(pts))
        for k, p in enumerate(rel):
            cosg = np.where(rs > 0, src @ p / np.where(rs > 0, rs, 1.0) / rp[k], 1.0)
            series[k] = plan.dV * sum(np.sum(rho * rs ** l * eval_legendre(l, cosg)) / rp[k] ** (l + 1)
                                      for l in range(l_max + 1))
        assert np.max(np.abs(vals - series)) < 1e-12 * np.abs(series).max()
        errs.append(np.max(np.abs(vals - coul)) / np.abs(coul).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-6


def test_multipole_solution_satisfies_the_extended_stencil():
    """phi = apply_fL_multipole(rho) solves the finite-difference equation on the
    grid extended by the exterior points, -L_full phi = 4 pi rho, with the
    stencil built from exact rational weights and the exterior values in place."""
    plan = oracle.Plan((12, 10, 14), (0.5, 0.55, 0.45), (D, D, D), U)
    c = oracle.expansion_centre(plan)
    rho = _gaussian(plan, c + np.array([0.2, 0.1, -0.3]), 2.5) - 0.5 * _gaussian(plan, c - 0.4, 5.0)
    l_max = 3
    phi = oracle.apply_fL_multipole(plan, rho, l_max)
    m = plan.fd_order // 2
    n1, n2, n3 = plan.n
    ext = np.zeros((n3 + 2 * m, n2 + 2 * m, n1 + 2 * m))
    ext[m:m + n3, m:m + n2, m:m + n1] = phi.reshape(n3, n2, n1)
    q = oracle.multipole_moments(plan, rho, l_max)
    for a, i_a, pts, flat in oracle.exterior_points(plan):
        vals = oracle.multipole_potential(plan, q, l_max, pts).reshape(
            [1 if b == a else plan.n[b] for b in (2, 1, 0)])
        sl = [slice(m, m + n3), slice(m, m + n2), slice(m, m + n1)]
        sl[2 - a] = slice(m + i_a, m + i_a + 1)
        ext[tuple(sl)] = vals
    w = [float(x) for x in exact_weights(plan.fd_order)]
    lap = np.zeros((n3, n2, n1))
    for a in range(3):
        for d in range(-m, m + 1):
            sl = [slice(m, m + n3), slice(m, m + n2), slice(m, m + n1)]
            sl[2 - a] = slice(m + d, m + d + plan.n[a])
            lap += w[abs(d)] / plan.h[a] ** 2 * ext[tuple(sl)]
    resid = -lap.ravel() - 4.0 * math.pi * rho
    assert np.max(np.abs(resid)) < 1e-10 * 4.0 * math.pi * np.abs(rho).max()


def test_multipole_boundary_reproduces_the_free_space_potential():
    """A normalised Gaussian charge in a Dirichlet box: with multipole boundary
    values the grid solution is the free-space potential erf(sqrt(a) r) / r up
    to the discretisation error everywhere, also next to the faces, where zero
    boundary values miss it by the whole 1/r tail."""
    from scipy.special import erf
    plan = oracle.Plan((24, 24, 24), (0.35,) * 3, (D, D, D), U)
    c = oracle.expansion_centre(plan)
    alpha = 3.0
    rho = _gaussian(plan, c, alpha)
    r = np.linalg.norm(oracle.interior_points(plan) - c, axis=1)
    exact = np.where(r > 0, erf(np.sqrt(alpha) * r) / np.where(r > 0, r, 1.0), 2.0 * np.sqrt(alpha / math.pi))
    err_mp = np.max(np.abs(oracle.apply_fL_multipole(plan, rho, 4) - exact)) / exact.max()
    err_zero = np.max(np.abs(oracle.apply_fL(plan, rho) - exact)) / exact.max()
    assert err_mp < 2e-4
    assert err_zero > 50 * err_mp


# ---------------------------------------------------------------- Bloch k-points (R13-R16)
def _complex_orbitals(rng, n_kpt, N, n_orb):
    return rng.standard_normal((n_kpt, N, n_orb)) + 1j * rng.standard_normal((n_kpt, N, n_orb))


@pytest.mark.parametrize("n,order,theta", [(9, 2, 0.7), (12, 12, -2.1), (7, 12, math.pi), (16, 8, 0.0),
                                           (5, 12, 1.3)])
def test_bloch_1d_plane_waves_and_eigenvalues(n, order, theta):
    """Every e^{i kappa x} with kappa = (2 pi m + theta) / n is an eigenvector of the
    Bloch matrix with the stencil's symbol as eigenvalue, also when the stencil
    wraps the cell more than once (n < order + 1)."""
    h = 0.37
    L = oracle.lap1d_bloch(n, h, order, theta)
    assert np.max(np.abs(L - L.conj().T)) < 1e-12 * np.abs(L).max()
    w = [float(x) for x in exact_weights(order)]
    x = np.arange(n)
    lam = []
    for m_ in range(n):
        kap = (2 * np.pi * m_ + theta) / n
        lk = (w[0] + 2 * sum(w[p] * np.cos(p * kap) for p in range(1, order // 2 + 1))) / h ** 2
        u = np.exp(1j * kap * x)
        assert np.max(np.abs(L @ u - lk * u)) < 1e-11 * abs(w[0]) / h ** 2
        lam.append(lk)
    assert np.max(np.abs(np.sort(lam) - np.linalg.eigvalsh(L))) < 1e-10 * abs(w[0]) / h ** 2
    if theta == 0.0:
        assert np.max(np.abs(L - oracle.lap1d(n, h, P, order))) == 0.0


@pytest.mark.parametrize("kind", [U, S])
def test_bloch_apply_fL_matches_dense_matrix_function(kind):
    """Mixed Bloch / Dirichlet axes: the Kronecker apply (complex Vk, conjugated
    forward contraction) equals f of the dense Hermitian 3D Laplacian."""
    base = oracle.Plan((5, 4, 6), (0.5, 0.45, 0.4), (P, D, P), kind, fd_order=4)
    theta = (0.9, 0.0, -2.4)
    bp = oracle.BlochPlan(base, theta)
    L1, L2, L3 = bp.L
    I1, I2, I3 = (np.eye(k) for k in base.n)
    Ld = np.kron(I3, np.kron(I2, L1)) + np.kron(I3, np.kron(L2, I1)) + np.kron(L3, np.kron(I2, I1))
    lam, V = np.linalg.eigh(Ld)
    mu = -lam
    fl = 4 * np.pi / mu if kind == U else 4 * np.pi * (1 - np.exp(-mu / (4 * 0.11 ** 2))) / mu
    F = (V * fl) @ V.conj().T
    rng = np.random.default_rng(5)
    b = rng.standard_normal(base.N) + 1j * rng.standard_normal(base.N)
    x = oracle.apply_fL_bloch(bp, b)
    assert np.max(np.abs(x - F @ b)) < 1e-11 * np.abs(F @ b).max()


def test_bloch_plane_wave_is_scaled_by_f():
    base = oracle.Plan((6, 5, 7), (0.4, 0.5, 0.45), (P, P, P), S)
    theta = (0.3, -1.1, 2.9)
    bp = oracle.BlochPlan(base, theta)
    w = [float(x) for x in exact_weights(12)]
    idx = np.indices((7, 5, 6))  # [x3, x2, x1]
    modes = (2, 4, 1)
    phase = np.zeros((7, 5, 6))
    lam = 0.0
    for a, (n, h, th, m_) in enumerate(zip(base.n, base.h, theta, modes)):
        kap = (2 * np.pi * m_ + th) / n
        phase = phase + kap * idx[2 - a]
        lam += (w[0] + 2 * sum(w[p] * np.cos(p * kap) for p in range(1, 7))) / h ** 2
    u = np.exp(1j * phase).ravel()
    f = 4 * np.pi * (1 - np.exp(lam / (4 * 0.11 ** 2))) / (-lam)
    assert np.max(np.abs(oracle.apply_fL_bloch(bp, u) - f * u)) < 1e-10 * f


def test_bloch_zero_phase_is_the_real_periodic_solve():
    base = oracle.Plan((6, 8, 5), (0.4, 0.35, 0.5), (P, P, D), U)
    b = np.random.default_rng(2).standard_normal(base.N)
    x = oracle.apply_fL_bloch(oracle.BlochPlan(base, (0.0, 0.0, 0.0)), b)
    ref = oracle.apply_fL(base, b)
    assert np.max(np.abs(x - ref)) < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("kind", [U, S])
def test_kpoint_exchange_is_the_supercell_exchange(kind):
    """k-point sampling along x1 with n_k phases 2 pi c / n_k is the Gamma-point
    exchange of the n_k-fold supercell whose orbitals are the Bloch orbitals
    continued cell by cell with their phase: with unit weights, Vx Psi on the
    first cell agrees and the supercell energy is n_k times the k-point sum.
    The supercell side uses a dense f from the independently derived stencil."""
    n_k = 3
    n1, n2, n3 = 4, 5, 4
    h = (0.45, 0.5, 0.4)
    base = oracle.Plan((n1, n2, n3), h, (P, P, D), kind, fd_order=6)
    theta = np.array([[2 * np.pi * c / n_k, 0.0, 0.0] for c in range(n_k)])
    rng = np.random.default_rng(17)
    n_orb = 2
    psi = _complex_orbitals(rng, n_k, base.N, n_orb)
    occ = rng.uniform(0.3, 1.0, (n_k, n_orb))
    wk = np.ones(n_k)
    vx, e = oracle.vx_kpoints(base, theta, wk, psi, occ)
    # supercell: cells c = 0..n_k-1 along x1, Psi(x1 + c n1) = e^{i c theta_q} psi_q(x1)
    sup = oracle.Plan((n_k * n1, n2, n3), h, (P, P, D), kind, fd_order=6)
    Ls = sparse_laplacian(sup).toarray()
    lam, V = np.linalg.eigh(Ls)
    mu = -lam
    fl = 4 * np.pi / mu if kind == U else 4 * np.pi * (1 - np.exp(-mu / (4 * 0.11 ** 2))) / mu
    F = (V * fl) @ V.T
    def unfold(u, th):
        cube = u.reshape(n3, n2, n1)
        return np.concatenate([np.exp(1j * c * th) * cube for c in range(n_k)], axis=2).ravel()
    Psi = [(q, m_, unfold(psi[q][:, m_], theta[q, 0])) for q in range(n_k) for m_ in range(n_orb)]
    e_sup = 0.0
    for k, n_, Pk in Psi:
        out = np.zeros(sup.N, dtype=complex)
        for q, m_, Pq in Psi:
            rho = np.conj(Pq) * Pk
            out -= occ[q, m_] * Pq * (F @ rho)
        first = out.reshape(n3, n2, n_k * n1)[:, :, :n1].ravel()
        assert np.max(np.abs(first - vx[k][:, n_])) < 1e-11 * np.abs(first).max()
        e_sup += 0.5 * base.dV * occ[k, n_] * np.vdot(Pk, out).real
    assert abs(e_sup - n_k * e) < 1e-11 * abs(e_sup)


def test_kpoint_energy_parseval_hermitian_and_negative():
    """E_x from <psi, Vx psi> equals the Parseval sum of Eq. 8; Vx is Hermitian
    (dV inner product) at each k-point; E_x < 0; and one k-point at theta = 0 with
    real orbitals is the Gamma-point exchange."""
    base = oracle.Plan((6, 4, 5), (0.4, 0.5, 0.45), (P, D, P), S, fd_order=8)
    rng = np.random.default_rng(23)
    theta = np.array([[0.0, 0.0, 0.0], [1.2, 0.0, -0.4], [-2.0, 0.0, 2.5]])
    wk = np.array([0.5, 0.3, 0.2])
    n_orb = 2
    psi = _complex_orbitals(rng, 3, base.N, n_orb)
    occ = rng.uniform(0.2, 1.0, (3, n_orb))
    vx, e = oracle.vx_kpoints(base, theta, wk, psi, occ)
    e_p = oracle.exchange_energy_kpoints(base, theta, wk, psi, occ)
    assert e < 0 and abs(e - e_p) < 1e-11 * abs(e)
    a = rng.standard_normal((base.N, 2)) + 1j * rng.standard_normal((base.N, 2))
    for k in range(3):
        va = oracle.vx_apply_kpoint(base, theta, wk, psi, occ, k, a)
        assert abs(np.vdot(a[:, 0], va[:, 1]) - np.conj(np.vdot(a[:, 1], va[:, 0]))) < 1e-11 * np.abs(va).max()
    psr = rng.standard_normal((base.N, 3))
    g = np.array([1.0, 0.5, 0.8])
    vx1, e1 = oracle.vx_kpoints(base, [[0.0, 0.0, 0.0]], [1.0], psr[None].astype(complex), g[None])
    vref, eref = oracle.vx_apply(base, psr, g)
    assert np.max(np.abs(vx1[0] - vref)) < 1e-12 * np.abs(vref).max()
    assert abs(e1 - eref) < 1e-12 * abs(eref)
