"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (stated once, used everywhere below):
  KX_FP64  : max-norm relative 1e-11 (float64 end to end; only summation order
             differs from the oracle).
  KX_F16X3 : Vx psi and f(L) b max-norm relative <= 1e-5, E_x relative <= 1e-6
             (the accuracy target of the split-precision path; each fp16 hi/lo
             product carries ~2^-22 relative error, six chained products plus fp32
             accumulation stay well inside these bounds).
"""
import numpy as np
import pytest

import oracle
import workloads
from workloads import DIRICHLET as D, PERIODIC as P, UNSCREENED as U, SCREENED as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: dict(vx=1e-11, ex=1e-11, fl=1e-11), 1: dict(vx=1e-5, ex=1e-6, fl=1e-5)}


@pytest.fixture(scope="module")
def kx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2406_16998_gb300 import build
    build.build()
    import paper_2406_16998_gb300 as k
    return k


def relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def system(n, h, bc, kind, n_orb, seed, centres=4):
    return workloads.System(n=n, h=h, bc=bc, kernel=kind, n_orb=n_orb, n_centres=centres, seed=seed)


# Grids chosen to span several 128-row tiles with ragged tails, padded K/N
# (sizes not multiples of 16), non-cubic shapes and mixed boundary conditions.
SMALL = [
    ((24, 40, 16), (0.45, 0.4, 0.5), (D, D, D), U, 5),
    ((16, 24, 48), (0.5, 0.5, 0.4), (P, P, D), U, 4),
    ((40, 32, 24), (0.4, 0.45, 0.5), (P, P, P), S, 4),
    ((8, 16, 8), (0.6, 0.5, 0.6), (D, P, D), S, 3),
    ((56, 8, 16), (0.3, 0.6, 0.5), (D, D, P), S, 2),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", range(len(SMALL)))
def test_vx_apply_matches_oracle(kx, prec, case):
    n, h, bc, kind, n_orb = SMALL[case]
    sysd = system(n, h, bc, kind, n_orb, 100 + case)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    vx = vx.cpu().numpy().T
    assert relmax(vx, vx_ref) < TOL[prec]["vx"]
    assert abs(ex.item() - ex_ref) < TOL[prec]["ex"] * abs(ex_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_only_and_occupations(kx, prec):
    n, h, bc, kind, n_orb = SMALL[0]
    sysd = system(n, h, bc, kind, n_orb, 7)
    psi = workloads.make_orbitals(sysd)
    occ = np.array([1.0, 0.9, 0.6, 0.35, 0.1])
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, ex_ref = oracle.vx_apply(op, psi, occ)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T), occ=dev(occ))
    e_only = kx.kx_energy(plan, dev(psi.T), occ=dev(occ))
    torch.cuda.synchronize()
    assert relmax(vx.cpu().numpy().T, vx_ref) < TOL[prec]["vx"]
    assert abs(ex.item() - ex_ref) < TOL[prec]["ex"] * abs(ex_ref)
    assert abs(e_only.item() - ex_ref) < TOL[prec]["ex"] * abs(ex_ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", [0, 2, 3])
def test_apply_fL_matches_oracle(kx, prec, case):
    n, h, bc, kind, _ = SMALL[case]
    op = oracle.Plan(n, h, bc, kind)
    B = workloads.random_field(op.N, 3, 9 + case)
    X_ref = oracle.apply_fL(op, B)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    X = kx.kx_apply_fL(plan, dev(B.T)).cpu().numpy().T
    for r in range(3):
        assert relmax(X[:, r], X_ref[:, r]) < TOL[prec]["fl"]


def test_fp64_odd_sizes(kx):
    n, h, bc = (7, 9, 11), (0.5, 0.45, 0.4), (D, P, D)
    sysd = system(n, h, bc, S, 3, 17)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, S)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, S, precision=0)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    assert relmax(vx.cpu().numpy().T, vx_ref) < 1e-11
    assert abs(ex.item() - ex_ref) < 1e-11 * abs(ex_ref)


def test_setup_eigendecomposition_and_ftable(kx):
    n, h, bc, kind = (24, 40, 16), (0.45, 0.4, 0.5), (D, P, D), S
    op = oracle.Plan(n, h, bc, kind)
    plan = kx.Plan(n, h, bc, kind, precision=1)
    for a in range(3):
        lam, V = plan.eig(a)
        L = oracle.lap1d(n[a], h[a], bc[a], 12)
        scale = np.abs(op.lam[a]).max()
        assert np.max(np.abs(lam - op.lam[a])) < 1e-12 * scale
        assert np.max(np.abs(L @ V - V * lam)) < 1e-12 * scale
        assert np.max(np.abs(V.T @ V - np.eye(n[a]))) < 1e-13
    f = plan.ftable()
    assert relmax(f, op.fdiag.reshape(-1)) < 1e-12


def test_single_orbital_and_tiny_grid(kx):
    n, h, bc = (8, 8, 8), (0.5,) * 3, (D, D, D)
    sysd = system(n, h, bc, U, 1, 23)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, U)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    for prec in (0, 1):
        plan = kx.Plan(n, h, bc, U, precision=prec)
        vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
        assert relmax(vx.cpu().numpy().T, vx_ref) < TOL[prec]["vx"]
        assert abs(ex.item() - ex_ref) < TOL[prec]["ex"] * abs(ex_ref)


@pytest.mark.parametrize("case", [0, 1, 2])
def test_fused_and_unfused_middle_passes(kx, case, monkeypatch):
    """The fused per-slice kernel (modes 2 and 1, f scaling, energy) and the
    three separate passes it replaces both match the oracle; the launch counts
    show which of the two ran."""
    n, h, bc, kind, n_orb = SMALL[case]
    sysd = system(n, h, bc, kind, n_orb, 200 + case)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, kind, precision=1)
    for fused in (True, False):
        monkeypatch.setenv("KX_SLAB", "1" if fused else "0")
        plan.profile(True)
        vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
        torch.cuda.synchronize()
        prof = plan.profile_read()
        plan.profile(False)
        assert plan.status() == kx.KX_OK
        assert (prof["slab"][1] > 0) == fused
        assert (prof["X2F"][1] > 0) == (not fused)
        assert prof["X3F"][1] > 0 and prof["X3I"][1] > 0
        assert relmax(vx.cpu().numpy().T, vx_ref) < TOL[1]["vx"]
        assert abs(ex.item() - ex_ref) < TOL[1]["ex"] * abs(ex_ref)


def test_max_axis_128(kx):
    n, h, bc = (128, 8, 16), (0.2, 0.5, 0.5), (D, P, D)
    sysd = system(n, h, bc, S, 2, 29)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, S)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, S, precision=1)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    assert relmax(vx.cpu().numpy().T, vx_ref) < 1e-5
    assert abs(ex.item() - ex_ref) < 1e-6 * abs(ex_ref)


def test_zero_orbital(kx):
    n, h, bc = (16, 16, 16), (0.5,) * 3, (D, D, D)
    sysd = system(n, h, bc, U, 2, 31)
    psi = workloads.make_orbitals(sysd)
    psi[:, 1] = 0.0
    op = oracle.Plan(n, h, bc, U)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, U, precision=1)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    vx = vx.cpu().numpy().T
    assert np.all(vx[:, 1] == 0.0)
    assert relmax(vx, vx_ref) < 1e-5 and abs(ex.item() - ex_ref) < 1e-6 * abs(ex_ref)


def test_ace_matches_oracle(kx):
    n, h, bc, kind, n_orb = SMALL[1]
    sysd = system(n, h, bc, kind, n_orb, 37)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, _ = oracle.vx_apply(op, psi)
    xi_ref, M_ref, _ = oracle.ace(op, psi, vx_ref)
    plan = kx.Plan(n, h, bc, kind, precision=0)
    xi, M = kx.kx_ace(plan, dev(psi.T), dev(vx_ref.T))
    assert relmax(M.cpu().numpy(), M_ref) < 1e-12
    assert relmax(xi.cpu().numpy().T, xi_ref) < 1e-10


# --------------------------------------------------------------------------
# Dirichlet values from the multipole expansion (isolated systems, Sec. 4)
# --------------------------------------------------------------------------
MP_GRID = ((16, 24, 24), (0.5, 0.45, 0.4), (D, D, D))


@pytest.mark.parametrize("prec,l_max", [(0, 0), (0, 2), (0, 4), (1, 2), (1, 4)])
def test_multipole_apply_fL_matches_oracle(kx, prec, l_max):
    n, h, bc = MP_GRID
    op = oracle.Plan(n, h, bc, U)
    b = workloads.random_field(op.N, 3, 71 + l_max)
    ref = np.stack([oracle.apply_fL_multipole(op, b[:, r], l_max) for r in range(3)], axis=1)
    plan = kx.Plan(n, h, bc, U, precision=prec)
    plan.set_multipole(l_max)
    x = kx.kx_apply_fL(plan, dev(b.T)).cpu().numpy().T
    assert relmax(x, ref) < (1e-11 if prec == 0 else TOL[1]["fl"])


@pytest.mark.parametrize("prec", [0, 1])
def test_multipole_vx_and_energy_match_oracle(kx, prec):
    n, h, bc = MP_GRID
    sysd = system(n, h, bc, U, 5, 73)
    psi = workloads.make_orbitals(sysd)
    occ = np.array([1.0, 0.9, 0.75, 0.5, 0.25])
    op = oracle.Plan(n, h, bc, U)
    vx_ref, ex_ref = oracle.vx_apply(op, psi, occ, l_max=3)
    vx0_ref, ex0_ref = oracle.vx_apply(op, psi, occ)
    plan = kx.Plan(n, h, bc, U, precision=prec)
    plan.set_multipole(3)
    psi_d, occ_d = dev(psi.T), dev(occ)
    vx, ex = kx.kx_vx_apply(plan, psi_d, occ_d)
    e_only = kx.kx_energy(plan, psi_d, occ_d)[0].item()
    tol = TOL[prec]
    assert relmax(vx.cpu().numpy().T, vx_ref) < tol["vx"]
    assert abs(ex.item() - ex_ref) < tol["ex"] * abs(ex_ref)
    assert abs(e_only - ex_ref) < tol["ex"] * abs(ex_ref)
    # the boundary values matter: the result differs from zero boundary values
    assert relmax(vx_ref, vx0_ref) > 1e-3
    plan.set_multipole(-1)
    vx0, ex0 = kx.kx_vx_apply(plan, psi_d, occ_d)
    assert relmax(vx0.cpu().numpy().T, vx0_ref) < tol["vx"]


@pytest.mark.parametrize("prec", [0, 1])
def test_multipole_pair_ranges_host_path_and_batch(kx, prec, monkeypatch):
    """With boundary values from the expansion: pair ranges add up to the full
    apply, the host-buffer entry point and a captured batch give the device
    path's result (the batch with the plan's launch shapes as they are: a tuned
    shape may take the separate middle passes, which round differently)."""
    from paper_2406_16998_gb300 import shard
    monkeypatch.setenv("KX_AUTOTUNE", "0")
    n, h, bc = MP_GRID
    psi = workloads.make_orbitals(system(n, h, bc, U, 6, 79))
    plan = kx.Plan(n, h, bc, U, precision=prec)
    plan.set_multipole(2)
    x = dev(psi.T)
    full, e_full = kx.kx_vx_apply(plan, x)
    acc = torch.zeros_like(full)
    e_acc = 0.0
    for r in range(3):
        a, b = shard.pair_range(6, r, 3)
        part, e_part = kx.kx_vx_apply_pairs(plan, x, a, b)
        acc += part
        e_acc += e_part.item()
    tol = 1e-12 if prec == 0 else 1e-6
    assert relmax(acc.cpu().numpy(), full.cpu().numpy()) < tol
    assert abs(e_acc - e_full.item()) < tol * abs(e_full.item())
    vx_h, ex_h = kx.kx_vx_apply_host(plan, torch.from_numpy(np.ascontiguousarray(psi.T)))
    assert np.array_equal(vx_h.numpy(), full.cpu().numpy()) and ex_h == e_full.item()
    out = torch.empty_like(full)
    ex_b = torch.empty(1, dtype=torch.float64, device="cuda")
    bt = kx.Batch([plan], [6])
    for _ in range(2):
        bt.run([x], [out], ex_b)
    torch.cuda.synchronize()
    bt.close()
    assert relmax(out.cpu().numpy(), full.cpu().numpy()) < 1e-12
    assert abs(ex_b.item() - e_full.item()) < 1e-12 * abs(e_full.item())


def test_multipole_rejects_unsupported_plans(kx):
    plan = kx.Plan((16, 16, 16), (0.5,) * 3, (P, P, D), U, precision=1)
    with pytest.raises(kx.KxError) as ei:
        plan.set_multipole(2)
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    plan = kx.Plan((16, 16, 16), (0.5,) * 3, (D, D, D), S, precision=1)
    with pytest.raises(kx.KxError) as ei:
        plan.set_multipole(2)
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    plan = kx.Plan((16, 16, 16), (0.5,) * 3, (D, D, D), U, precision=1)
    with pytest.raises(kx.KxError) as ei:
        plan.set_multipole(9)
    assert ei.value.code == kx.KX_ERR_ARG
    plan.set_multipole(1)
    b = dev(workloads.random_field(plan.N, 1, 3).T)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_apply_fL_noalloc(plan, b, torch.empty_like(b))
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED



@pytest.mark.parametrize("prec", [0, 1])
def test_multipole_energy_gradient_against_finite_differences(kx, prec):
    """dE_x/dpsi with multipole boundary values (the solve is not symmetric in
    rho) against central finite differences of the oracle's E_x, and the
    autograd energy's backward against the same gradient."""
    n, h, bc = MP_GRID
    sysd = system(n, h, bc, U, 3, 97)
    psi = workloads.make_orbitals(sysd)
    occ = np.array([1.0, 0.7, 0.4])
    op = oracle.Plan(n, h, bc, U)
    plan = kx.Plan(n, h, bc, U, precision=prec)
    plan.set_multipole(2)
    psi_d, occ_d = dev(psi.T), dev(occ)
    grad, ex = kx.kx_energy_gradient(plan, psi_d, occ_d)
    grad = grad.cpu().numpy().T
    _, ex_ref = oracle.vx_apply(op, psi, occ, l_max=2)
    assert abs(ex.item() - ex_ref) < TOL[prec]["ex"] * abs(ex_ref)
    rng = np.random.default_rng(11)
    step = 1e-4
    scale = np.abs(grad).max()
    for _ in range(6):
        r, k = int(rng.integers(op.N)), int(rng.integers(3))
        pp, pm = psi.copy(), psi.copy()
        pp[r, k] += step
        pm[r, k] -= step
        fd = (oracle.vx_apply(op, pp, occ, l_max=2)[1] - oracle.vx_apply(op, pm, occ, l_max=2)[1]) / (2 * step)
        assert abs(fd - grad[r, k]) < (1e-7 if prec == 0 else 1e-5) * scale
    # the gradient is not 2 dV g Vx psi here (that would use the solve, not its symmetric part)
    vx, _ = kx.kx_vx_apply(plan, psi_d, occ_d)
    naive = 2 * sysd.dV * vx.cpu().numpy().T * occ[None, :]
    assert relmax(naive, grad) > 1e-4
    x = psi_d.clone().requires_grad_(True)
    e = kx.exchange_energy(x, plan, occ_d)
    e.backward()
    assert relmax(x.grad.cpu().numpy().T, grad) < 1e-12


def test_energy_gradient_is_2dv_vx_with_zero_boundary_values(kx):
    n, h, bc, kind, n_orb = SMALL[0]
    psi = workloads.make_orbitals(system(n, h, bc, kind, n_orb, 99))
    plan = kx.Plan(n, h, bc, kind, precision=1)
    psi_d = dev(psi.T)
    grad, ex = kx.kx_energy_gradient(plan, psi_d)
    vx, ex2 = kx.kx_vx_apply(plan, psi_d)
    assert np.array_equal(grad.cpu().numpy(), (2 * plan.dV * vx).cpu().numpy())
    assert ex.item() == ex2.item()


def test_multipole_more_than_64_orbitals(kx):
    """Tensor-core plans with more than 64 orbitals take the CUDA-core form of
    the multipole correction (weighted projections, FMA combination applied
    to Vx psi after the pair loop): a pair range of a 70-orbital system
    against the oracle over the same pairs."""
    from paper_2406_16998_gb300 import shard
    n, h, bc = (16, 16, 24), (0.55, 0.55, 0.5), (D, D, D)
    sysd = system(n, h, bc, U, 70, 101, centres=6)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, U)
    plan = kx.Plan(n, h, bc, U, precision=1)
    plan.set_multipole(2)
    part, e_part = kx.kx_vx_apply_pairs(plan, dev(psi.T), 0, 40)
    ref, e_ref = oracle.vx_apply(op, psi, pairs=shard.pair_list(70)[:40], l_max=2)
    assert relmax(part.cpu().numpy().T, ref) < TOL[1]["vx"]
    assert abs(e_part.item() - e_ref) < TOL[1]["ex"] * abs(e_ref)


def test_full_size_apply_is_deterministic(kx):
    """Two applies of the benchmark system give bit-identical Vx psi and E_x
    (fixed-order reductions, no floating-point atomics)."""
    sysd = workloads.C2
    psi = dev(workloads.make_orbitals(sysd).T)
    plan = kx.Plan.for_system(sysd, precision=1)
    a, ea = kx.kx_vx_apply(plan, psi)
    b, eb = kx.kx_vx_apply(plan, psi)
    assert torch.equal(a, b) and ea.item() == eb.item()


def test_multipole_full_size_row(kx):
    """The 96^3 / 64-orbital benchmark system with boundary values to order 4,
    in the launch configuration of the benchmark: one orbital's row of pair
    solves against the oracle, and E_x through 1/2 sum_i dV <psi_i, (Vx psi)_i>."""
    sysd = workloads.C2
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    plan = kx.Plan.for_system(sysd, precision=1)
    plan.set_multipole(4)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    vx_h = vx.cpu().numpy()
    assert abs(ex.item() - 0.5 * sysd.dV * np.einsum("ij,ij->", psi.T, vx_h)) < 1e-6 * abs(ex.item())
    i = 5
    pairs = [(i, j) for j in range(psi.shape[1])]
    ref, _ = oracle.vx_apply(op, psi, ordered=True, pairs=pairs, l_max=4)
    # the row's error against the row's own scale
    assert np.max(np.abs(vx_h[i] - ref[:, i])) < 1e-5 * np.abs(ref[:, i]).max()


# --------------------------------------------------------------------------
# FFT variant for fully periodic grids (KX_FFT32)
# --------------------------------------------------------------------------
# (axes of 80 points take the register four-step path, 16 x 5, on each axis in turn)
@pytest.mark.parametrize("n", [(20, 24, 30), (16, 15, 18), (9, 10, 12), (80, 9, 10), (12, 80, 9), (10, 12, 80)])
def test_fft_apply_fL_matches_oracle(kx, n):
    h, bc = (0.45, 0.5, 0.4), (P, P, P)
    op = oracle.Plan(n, h, bc, S)
    b = workloads.random_field(op.N, 3, 83)
    ref = np.stack([oracle.apply_fL(op, b[:, r]) for r in range(3)], axis=1)
    plan = kx.Plan(n, h, bc, S, precision=kx.KX_FFT32)
    x = kx.kx_apply_fL(plan, dev(b.T)).cpu().numpy().T
    assert relmax(x, ref) < TOL[1]["fl"]


def test_fft_vx_and_energy_match_oracle(kx):
    n, h, bc = (24, 20, 18), (0.45, 0.5, 0.4), (P, P, P)
    sysd = system(n, h, bc, S, 5, 89)
    psi = workloads.make_orbitals(sysd)
    occ = np.array([1.0, 0.8, 0.6, 0.4, 0.2])
    op = oracle.Plan(n, h, bc, S)
    vx_ref, ex_ref = oracle.vx_apply(op, psi, occ)
    plan = kx.Plan(n, h, bc, S, precision=kx.KX_FFT32)
    psi_d, occ_d = dev(psi.T), dev(occ)
    vx, ex = kx.kx_vx_apply(plan, psi_d, occ_d)
    e_only = kx.kx_energy(plan, psi_d, occ_d)[0].item()
    assert relmax(vx.cpu().numpy().T, vx_ref) < TOL[1]["vx"]
    assert abs(ex.item() - ex_ref) < TOL[1]["ex"] * abs(ex_ref)
    assert abs(e_only - ex_ref) < TOL[1]["ex"] * abs(ex_ref)


def test_fft_rejects_unsupported_grids(kx):
    with pytest.raises(kx.KxError) as ei:
        kx.Plan((16, 16, 16), (0.5,) * 3, (P, P, D), S, precision=kx.KX_FFT32)
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    with pytest.raises(kx.KxError) as ei:
        kx.Plan((14, 16, 16), (0.5,) * 3, (P, P, P), S, precision=kx.KX_FFT32)  # 14 = 2 x 7
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    with pytest.raises(kx.KxError) as ei:
        kx.Plan((8, 8, 160), (0.5,) * 3, (P, P, P), S, precision=kx.KX_FFT32)  # 160 > 128 points
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    plan = kx.Plan((16, 16, 16), (0.5,) * 3, (P, P, P), S, precision=kx.KX_FFT32)
    b = dev(workloads.random_field(plan.N, 1, 3).T)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_apply_fL_noalloc(plan, b, torch.empty_like(b))
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED


def test_fft_full_size_against_kronecker_and_oracle(kx):
    """The 80^3 periodic screened 256-orbital system: the FFT plan's first 12
    pairs against the oracle, and its full apply against the tensor-core
    Kronecker plan on the same orbitals (both are f(L) on the same grid)."""
    sysd = workloads.C3
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    plan = kx.Plan.for_system(sysd, precision=kx.KX_FFT32)
    psi_d = dev(psi.T)
    part, e_part = kx.kx_vx_apply_pairs(plan, psi_d, 0, 12)
    from paper_2406_16998_gb300 import shard
    ref, e_ref = oracle.vx_apply(op, psi, pairs=shard.pair_list(psi.shape[1])[:12])
    assert relmax(part.cpu().numpy().T, ref) < 1e-5
    assert abs(e_part.item() - e_ref) < 1e-6 * abs(e_ref)
    vx_f, ex_f = kx.kx_vx_apply(plan, psi_d)
    vx_k, ex_k = kx.kx_vx_apply(kx.Plan.for_system(sysd, precision=1), psi_d)
    assert relmax(vx_f.cpu().numpy(), vx_k.cpu().numpy()) < 2e-5
    assert abs(ex_f.item() - ex_k.item()) < 2e-6 * abs(ex_k.item())


def test_ace_f16x3_plan_matches_oracle(kx):
    """The tensor-core plan's ACE tail: float32 products, float64 block sums and
    float64 Cholesky; M to 1e-6 and xi to 1e-5 of their largest entries."""
    n, h, bc, kind, n_orb = SMALL[1]
    sysd = system(n, h, bc, kind, n_orb, 37)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, _ = oracle.vx_apply(op, psi)
    xi_ref, M_ref, _ = oracle.ace(op, psi, vx_ref)
    plan = kx.Plan(n, h, bc, kind, precision=1)
    xi, M = kx.kx_ace(plan, dev(psi.T), dev(vx_ref.T))
    assert relmax(M.cpu().numpy(), M_ref) < 1e-6
    assert relmax(xi.cpu().numpy().T, xi_ref) < 1e-5


# n (grid), precision, n_xi, n_vec: ragged grids (float64 plan), several
# projection and combination tiles, single vectors
ACE_APPLY_CASES = [
    ((13, 11, 7), 0, 1, 1),
    ((13, 11, 7), 0, 7, 33),
    ((24, 40, 16), 0, 65, 70),
    ((24, 40, 16), 1, 1, 1),
    ((24, 40, 16), 1, 7, 33),
    ((24, 40, 16), 1, 64, 64),
    ((32, 16, 40), 1, 65, 130),
    ((16, 8, 8), 1, 200, 3),
]


@pytest.mark.parametrize("n,prec,n_xi,n_vec", ACE_APPLY_CASES)
def test_ace_apply_matches_oracle(kx, n, prec, n_xi, n_vec):
    """-xi (dV xi^T phi) on seeded inputs against the float64 oracle: 1e-12 for
    float64 plans, 2e-6 (float32 products) for tensor-core plans."""
    h, bc = (0.4, 0.45, 0.5), (D, P, D)
    op = oracle.Plan(n, h, bc, U)
    xi = workloads.random_field(op.N, n_xi, 101 + n_xi) * 0.3
    phi = workloads.random_field(op.N, n_vec, 202 + n_vec)
    ref = oracle.ace_apply(op, xi, phi)
    plan = kx.Plan(n, h, bc, U, precision=prec)
    out = kx.kx_ace_apply(plan, dev(xi.T), dev(phi.T))
    tol = 1e-12 if prec == 0 else 2e-6
    assert relmax(out.cpu().numpy().T, ref) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_ace_operator_reproduces_vx_on_orbitals(kx, prec):
    """kx_ace then kx_ace_apply on the orbitals gives back Vx psi (the property
    the compressed operator is built for), against the oracle's pair-by-pair Vx."""
    n, h, bc, kind, n_orb = SMALL[2]
    sysd = system(n, h, bc, kind, n_orb, 43)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    vx_ref, _ = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    psi_d = dev(psi.T)
    xi, _ = kx.kx_ace(plan, psi_d, dev(vx_ref.T))
    out = kx.kx_ace_apply(plan, xi, psi_d)
    assert relmax(out.cpu().numpy().T, vx_ref) < (1e-10 if prec == 0 else 1e-5)


def test_ace_apply_unaligned_inputs(kx):
    """Inputs that start 8 bytes off a 16-byte boundary take the 8-byte copy
    path of the float32 kernels and give the same result as aligned ones."""
    n, h, bc = (24, 40, 16), (0.4, 0.45, 0.5), (D, P, D)
    op = oracle.Plan(n, h, bc, U)
    xi = workloads.random_field(op.N, 9, 5) * 0.3
    phi = workloads.random_field(op.N, 5, 6)
    plan = kx.Plan(n, h, bc, U, precision=1)
    ref = kx.kx_ace_apply(plan, dev(xi.T), dev(phi.T)).cpu().numpy()

    def shifted(a):
        flat = torch.zeros(a.size + 1, dtype=torch.float64, device="cuda")
        flat[1:] = dev(a.reshape(-1))
        return flat[1:].view(a.shape)

    xs, ps = shifted(np.ascontiguousarray(xi.T)), shifted(np.ascontiguousarray(phi.T))
    assert xs.data_ptr() % 16 == 8 and ps.data_ptr() % 16 == 8
    out = kx.kx_ace_apply(plan, xs, ps).cpu().numpy()
    assert np.array_equal(out, ref)
    assert relmax(out.T, oracle.ace_apply(op, xi, phi)) < 2e-6


def test_ace_apply_rejects_bad_arguments(kx):
    n, h, bc = (16, 8, 8), (0.5,) * 3, (D, D, D)
    plan = kx.Plan(n, h, bc, U, precision=1)
    xi = dev(workloads.random_field(plan.N, 3, 1).T)
    phi = dev(workloads.random_field(plan.N, 2, 2).T)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_ace_apply(plan, xi, phi, out=phi)  # out overlaps phi
    assert ei.value.code == kx.KX_ERR_ARG
    with pytest.raises(kx.KxError) as ei:
        kx.kx_ace_apply(plan, xi, phi, out=xi[:2])  # out overlaps xi
    assert ei.value.code == kx.KX_ERR_ARG
    big = dev(workloads.random_field(plan.N, 257, 3).T)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_ace_apply(plan, big, phi)
    assert ei.value.code == kx.KX_ERR_ARG


def test_batch_follows_plan_changes(kx):
    """A batch's captured graph refers to its plans' buffers: after the plan is
    used with another pair range (its pair list is rebuilt) or switched to
    multipole boundary values, the next run captures again and still gives
    the direct result."""
    n, h, bc = MP_GRID
    psi = workloads.make_orbitals(system(n, h, bc, U, 6, 103))
    plan = kx.Plan(n, h, bc, U, precision=1)
    x = dev(psi.T)
    out = torch.empty_like(x)
    ex = torch.empty(1, dtype=torch.float64, device="cuda")
    b = kx.Batch([plan], [6])
    b.run([x], [out], ex)
    ref0, _ = kx.kx_vx_apply(plan, x)
    torch.cuda.synchronize()
    assert relmax(out.cpu().numpy(), ref0.cpu().numpy()) < 1e-12
    kx.kx_vx_apply_pairs(plan, x, 3, 9)  # rebuilds the plan's pair list for a sub-range
    b.run([x], [out], ex)
    torch.cuda.synchronize()
    assert relmax(out.cpu().numpy(), ref0.cpu().numpy()) < 1e-12
    plan.set_multipole(2)
    ref1, e1 = kx.kx_vx_apply(plan, x)
    b.run([x], [out], ex)
    torch.cuda.synchronize()
    assert relmax(out.cpu().numpy(), ref1.cpu().numpy()) < 1e-12
    assert abs(ex.item() - e1.item()) < 1e-12 * abs(e1.item())
    assert relmax(ref1.cpu().numpy(), ref0.cpu().numpy()) > 1e-3
    b.close()


def test_batch_equals_individual_runs(kx):
    cases = [SMALL[0], SMALL[2], SMALL[3]]
    plans, psis, refs = [], [], []
    for c, (n, h, bc, kind, n_orb) in enumerate(cases):
        sysd = system(n, h, bc, kind, n_orb, 41 + c)
        psi = workloads.make_orbitals(sysd)
        plans.append(kx.Plan(n, h, bc, kind, precision=1))
        psis.append(dev(psi.T))
        refs.append(oracle.vx_apply(oracle.Plan(n, h, bc, kind), psi))
    outs = [torch.empty_like(p) for p in psis]
    ex = torch.empty(len(cases), dtype=torch.float64, device="cuda")
    b = kx.Batch(plans, [p.shape[0] for p in psis])
    for _ in range(2):  # second run replays the captured graph
        b.run(psis, outs, ex)
    torch.cuda.synchronize()
    for k, (vx_ref, ex_ref) in enumerate(refs):
        single, e1 = kx.kx_vx_apply(plans[k], psis[k])
        assert relmax(outs[k].cpu().numpy().T, vx_ref) < 1e-5
        assert abs(ex[k].item() - ex_ref) < 1e-6 * abs(ex_ref)
        assert relmax(outs[k].cpu().numpy(), single.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_matches_oracle_gradient(kx, prec):
    n, h, bc, kind, n_orb = SMALL[3]
    sysd = system(n, h, bc, kind, n_orb, 43)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    g_ref = oracle.energy_gradient(op, psi)
    e_ref = oracle.exchange_energy(op, psi)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    x = dev(psi.T).requires_grad_(True)
    e = kx.exchange_energy(x, plan)
    e.backward()
    assert abs(e.item() - e_ref) < TOL[prec]["ex"] * abs(e_ref)
    assert relmax(x.grad.cpu().numpy().T, g_ref) < TOL[prec]["vx"]


def test_autograd_central_differences_fp64(kx):
    n, h, bc, kind, n_orb = (8, 16, 8), (0.6, 0.5, 0.6), (D, P, D), S, 3
    sysd = system(n, h, bc, kind, n_orb, 47)
    psi = workloads.make_orbitals(sysd)
    plan = kx.Plan(n, h, bc, kind, precision=0)
    x = dev(psi.T).requires_grad_(True)
    kx.exchange_energy(x, plan).backward()
    grad = x.grad.cpu().numpy()
    rng = np.random.default_rng(3)
    step = 1e-4
    for _ in range(16):
        k, r = int(rng.integers(n_orb)), int(rng.integers(plan.N))
        pp = psi.T.copy()
        pm = psi.T.copy()
        pp[k, r] += step
        pm[k, r] -= step
        ep = kx.kx_energy(plan, dev(pp)).item()
        em = kx.kx_energy(plan, dev(pm)).item()
        fd = (ep - em) / (2 * step)
        assert abs(fd - grad[k, r]) < 1e-7 * np.abs(grad).max()


def test_failure_paths(kx, monkeypatch):
    # bounded wait that nothing completes: the kernel gives up, status reports the timeout
    plan = kx.Plan((8, 8, 8), (0.5,) * 3, (D, D, D), U, precision=1)
    assert plan.status() == kx.KX_OK
    kx.kx_selftest_wait(plan, 2_000_000)
    assert plan.status() == kx.KX_ERR_TIMEOUT
    assert plan.status() == kx.KX_OK  # cleared by the read
    # the context is still usable afterwards
    psi = workloads.make_orbitals(system((8, 8, 8), (0.5,) * 3, (D, D, D), U, 2, 53))
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    assert np.isfinite(ex.item())
    # injected allocation failure on a fresh plan
    monkeypatch.setenv("KX_FAULT", "alloc")
    plan2 = kx.Plan((8, 8, 8), (0.5,) * 3, (D, D, D), U, precision=1)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_vx_apply(plan2, dev(psi.T))
    assert ei.value.code == kx.KX_ERR_NOMEM
    monkeypatch.delenv("KX_FAULT")
    kx.kx_vx_apply(plan2, dev(psi.T))
    # singular request
    with pytest.raises(kx.KxError) as ei:
        kx.Plan((8, 8, 8), (0.5,) * 3, (P, P, P), U)
    assert ei.value.code == kx.KX_ERR_SINGULAR
    # shape checks in the binding
    with pytest.raises(ValueError):
        kx.kx_vx_apply(plan, dev(psi.T[:, :-8]))


# --------------------------------------------------------------------------
# Full-size workloads, in the launch configuration the benchmark times:
# sampled orbitals against the oracle (one orbital's row of pair solves), and
# E_x through the identity E_x = 1/2 sum_i g_i dV <psi_i, (Vx psi)_i>.
# --------------------------------------------------------------------------
def _row_reference(op, psi, i):
    pairs = [(i, j) for j in range(psi.shape[1])]
    vx, _ = oracle.vx_apply(op, psi, ordered=True, pairs=pairs)
    return vx[:, i]


@pytest.mark.parametrize("name,sample", [("C2", (0, 37)), ("C3", (5,))])
def test_full_size_sampled(kx, name, sample):
    sysd = getattr(workloads, name)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    plan = kx.Plan.for_system(sysd, precision=1)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    vx_h = vx.cpu().numpy()
    M_diag = sysd.dV * np.einsum("ij,ij->i", psi.T, vx_h)
    assert abs(ex.item() - 0.5 * M_diag.sum()) < 1e-6 * abs(ex.item())
    for i in sample:
        ref = _row_reference(op, psi, i)
        # each sampled row against its own largest entry
        assert np.max(np.abs(vx_h[i] - ref)) < 1e-5 * np.abs(ref).max()


def test_full_size_pair_range_against_oracle(kx):
    """The benchmark system (96^3, 64 orbitals) on the tensor-core plan over the
    first 260 pairs of the library's pair list (the sample the benchmark's
    oracle leg times): partial Vx psi and partial E_x against the oracle's sums
    over the same pairs, at the split-path tolerances."""
    from paper_2406_16998_gb300 import shard
    sysd = workloads.C2
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    n_pairs = 260
    ref, e_ref = oracle.vx_apply(op, psi, pairs=shard.pair_list(sysd.n_orb)[:n_pairs])
    plan = kx.Plan.for_system(sysd, precision=1)
    part, e_part = kx.kx_vx_apply_pairs(plan, dev(psi.T), 0, n_pairs)
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    got = part.cpu().numpy().T
    assert relmax(got, ref) < TOL[1]["vx"]
    assert abs(e_part.item() - e_ref) < TOL[1]["ex"] * abs(e_ref)


def test_ace_full_size(kx):
    """The ACE tail and the compressed operator at the benchmark's size (96^3,
    64 orbitals, tensor-core plan) against the oracle on the whole output:
    W = -psi S with S symmetric positive definite (so -M is), xi from the
    oracle's construction as the apply's input."""
    sysd = workloads.C2
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega)
    rng = np.random.default_rng(77)
    Q, _ = np.linalg.qr(rng.standard_normal((sysd.n_orb, sysd.n_orb)))
    S_mat = (Q * rng.uniform(0.5, 2.0, sysd.n_orb)) @ Q.T
    W = -psi @ S_mat
    xi_ref, M_ref, _ = oracle.ace(op, psi, W)
    ref = oracle.ace_apply(op, xi_ref, psi)
    plan = kx.Plan.for_system(sysd, precision=1)
    psi_d = dev(psi.T)
    xi, M = kx.kx_ace(plan, psi_d, dev(W.T))
    assert relmax(M.cpu().numpy(), M_ref) < 1e-6
    assert relmax(xi.cpu().numpy().T, xi_ref) < 1e-5
    out = kx.kx_ace_apply(plan, dev(xi_ref.T), psi_d)
    assert relmax(out.cpu().numpy().T, ref) < 2e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_pair_ranges_sum_to_full_apply(kx, prec):
    from paper_2406_16998_gb300 import shard
    n, h, bc, kind, n_orb = SMALL[0]
    psi = workloads.make_orbitals(system(n, h, bc, kind, n_orb, 59))
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    x = dev(psi.T)
    full, e_full = kx.kx_vx_apply(plan, x)
    acc = torch.zeros_like(full)
    e_acc = 0.0
    for r in range(3):
        a, b = shard.pair_range(n_orb, r, 3)
        part, e_part = kx.kx_vx_apply_pairs(plan, x, a, b)
        acc += part
        e_acc += e_part.item()
    tol = 1e-12 if prec == 0 else 1e-6
    assert relmax(acc.cpu().numpy(), full.cpu().numpy()) < tol
    assert abs(e_acc - e_full.item()) < tol * abs(e_full.item())


@pytest.mark.parametrize("prec", [0, 1])
def test_host_buffers_match_device_path(kx, prec, monkeypatch):
    """kx_vx_apply_host (host buffers; the orbitals copied in pieces that the
    first chunks start on, rows of Vx psi copied back chunk by chunk as they
    become final) gives the device path's Vx psi bit for bit, over several
    chunks of the pair list; E_x to the last bits (the host path cuts its chunks
    at the copy pieces, which regroups the float64 energy sum)."""
    monkeypatch.setenv("KX_CHUNK_PAIRS", "16")
    n, h, bc = (24, 16, 32), (0.4, 0.45, 0.5), (D, P, D)
    sysd = system(n, h, bc, S, 12, 61)
    psi = workloads.make_orbitals(sysd)
    plan = kx.Plan(n, h, bc, S, precision=prec)
    psi_d = dev(psi.T)
    vx, ex = kx.kx_vx_apply(plan, psi_d)
    vx = vx.cpu().numpy()
    for pinned in (False, True):
        psi_h = torch.from_numpy(np.ascontiguousarray(psi.T))
        if pinned:
            psi_h = psi_h.pin_memory()
        vx_h, ex_h = kx.kx_vx_apply_host(plan, psi_h)
        assert plan.status() == kx.KX_OK
        assert np.array_equal(vx_h.numpy(), vx)
        assert abs(ex_h - ex.item()) <= 1e-13 * abs(ex.item())


def test_unaligned_output_pointer(kx):
    """An output that is 8- but not 16-byte aligned takes the scalar final pass
    and gives the same values."""
    import ctypes
    n, h, bc = (16, 24, 16), (0.5, 0.4, 0.5), (D, D, D)
    sysd = system(n, h, bc, U, 5, 62)
    psi = workloads.make_orbitals(sysd)
    plan = kx.Plan(n, h, bc, U, precision=1)
    psi_d = dev(psi.T)
    vx, _ = kx.kx_vx_apply(plan, psi_d)
    n_orb, N = psi_d.shape
    buf = torch.empty(n_orb * N + 1, dtype=torch.float64, device="cuda")
    ex = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = kx.lib().kx_vx_apply(plan.handle, n_orb, ctypes.c_void_p(psi_d.data_ptr()), None,
                              ctypes.c_void_p(buf.data_ptr() + 8), ctypes.c_void_p(ex.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == kx.KX_OK
    assert torch.equal(buf[1:].view(n_orb, N), vx)


def test_autotune_then_apply(kx):
    """kx_autotune times the launch shapes on synthetic orbitals and keeps one;
    the apply afterwards still matches the oracle."""
    n, h, bc = (24, 16, 32), (0.4, 0.45, 0.5), (D, P, D)
    sysd = system(n, h, bc, S, 6, 63)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, S)
    vx_ref, ex_ref = oracle.vx_apply(op, psi)
    plan = kx.Plan(n, h, bc, S, precision=1)
    assert plan.tuning()["tuned_ms"] == 0.0
    kx.kx_autotune(plan, 6, 200)
    t = plan.tuning()
    assert t["tuned_ms"] > 0.0 and t["fuse_slab"] in (0, 1) and t["pass_stages"] in (0, 2)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T))
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    assert relmax(vx.cpu().numpy().T, vx_ref) < TOL[1]["vx"]
    assert abs(ex.item() - ex_ref) < TOL[1]["ex"] * abs(ex_ref)
    # a second plan of the same shape takes the choice from the process-wide table
    plan2 = kx.Plan(n, h, bc, S, precision=1)
    kx.kx_autotune(plan2, 6, 200)
    assert plan2.tuning() == t
    # every candidate shape gives the same result within the split tolerance
    for fz, st in ((0, 2), (1, 0)):
        import os
        os.environ["KX_SLAB"] = str(fz)
        try:
            vx2, _ = kx.kx_vx_apply(plan2, dev(psi.T))
        finally:
            del os.environ["KX_SLAB"]
        assert relmax(vx2.cpu().numpy().T, vx_ref) < TOL[1]["vx"]


# ---------------------------------------------------------------- Bloch k-points
# Complex float32 mode products (plans other than KX_FP64): each of the six
# products sums n float32 terms (relative error ~n 2^-24), so Vx psi is held to
# 2e-5 of its largest entry and E_x (a float64 sum of many such values) to 2e-6.
TOL_K = {0: (1e-11, 1e-11), 1: (2e-5, 2e-6), 2: (2e-5, 2e-6)}
KPOINT_CASES = [
    # n, h, bc, kind, n_orb, k-grid, phase shift, precision
    ((12, 10, 14), (0.45, 0.5, 0.4), (P, P, D), U, 3, (2, 2, 1), (0.0, 0.0), 0),   # slab
    ((16, 8, 16), (0.45, 0.5, 0.4), (P, P, D), U, 3, (2, 2, 1), (0.0, 0.0), 1),
    ((10, 12, 9), (0.5, 0.45, 0.5), (P, P, P), S, 2, (3, 1, 1), (0.4, -0.3), 0),  # bulk, shifted grid
    ((10, 12, 9), (0.5, 0.45, 0.5), (P, P, P), S, 2, (3, 1, 1), (0.4, -0.3), 2),
    ((9, 20, 11), (0.5, 0.4, 0.5), (D, P, D), U, 3, (1, 3, 1), (0.0, 0.0), 0),    # wire
    ((8, 24, 16), (0.5, 0.4, 0.5), (D, P, D), S, 2, (1, 3, 1), (0.0, 0.0), 1),
    ((100, 6, 5), (0.3, 0.5, 0.5), (P, D, D), U, 2, (2, 1, 1), (0.0, 0.0), 0),    # several column splits
    ((128, 8, 8), (0.3, 0.5, 0.5), (P, D, D), S, 2, (2, 1, 1), (0.0, 0.0), 1),
    # axes of 32 and 64 points take the tensor-core products on float32 plans
    ((32, 16, 64), (0.45, 0.5, 0.4), (P, P, D), U, 3, (2, 2, 1), (0.0, 0.0), 1),
    ((64, 32, 8), (0.3, 0.4, 0.5), (P, D, P), S, 2, (2, 1, 2), (0.3, 0.1), 1),
    # 64 pencils per item: 128-pencil tensor-core tiles straddle two items, and
    # 9 pairs leave a ragged last tile (first product, and the f-scaled third)
    ((64, 8, 8), (0.3, 0.5, 0.5), (P, D, D), U, 3, (2, 1, 1), (0.0, 0.0), 1),
    ((8, 8, 64), (0.5, 0.5, 0.3), (D, D, P), S, 3, (1, 1, 3), (0.0, 0.0), 1),
    # every axis of 32 or 64 points: axes 2 and 3 take the pass kernel with
    # per-item scales, and with 64 points along axis 1 that axis does too
    ((32, 32, 32), (0.4, 0.45, 0.5), (P, P, D), U, 3, (2, 2, 1), (0.2, -0.1), 1),
    ((64, 32, 32), (0.3, 0.4, 0.5), (P, D, P), S, 2, (2, 1, 2), (0.0, 0.3), 1),
]


def kpoint_inputs(case, seed):
    n, h, bc, kind, n_orb, counts, shift, prec = KPOINT_CASES[case]
    sysd = system(n, h, bc, kind, n_orb, seed)
    theta, wk = workloads.kpoint_grid(sysd, counts)
    theta[:, 0] += shift[0] if bc[0] == P else 0.0
    theta[:, 1] += shift[1] if bc[1] == P else 0.0
    psi = workloads.make_bloch_orbitals(sysd, theta)
    occ = np.random.default_rng(seed).uniform(0.3, 1.0, (len(wk), n_orb))
    return sysd, theta, wk, psi, occ, prec


def to_dev_orbitals(psi):
    return dev(np.transpose(psi, (0, 2, 1)))  # (n_kpt, n_orb, N) complex128


@pytest.mark.parametrize("case", range(len(KPOINT_CASES)))
def test_kpoint_vx_and_energy_match_oracle(kx, case):
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(case, 300 + case)
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel)
    vx_ref, ex_ref = oracle.vx_kpoints(base, theta, wk, psi, occ)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    plan.profile(True)
    vx, ex = kx.kx_vx_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ))
    torch.cuda.synchronize()
    prof = plan.profile_read()
    vx = vx.cpu().numpy().transpose(0, 2, 1)
    assert relmax(vx, vx_ref) < TOL_K[prec][0]
    assert abs(ex.item() - ex_ref) < TOL_K[prec][1] * abs(ex_ref)
    n_k = len(wk)
    # six mode products per k-point pair block (k, q), q >= k (the reversed
    # blocks reuse the same solves, conjugated), one chunk each
    assert prof["bloch"][1] == 6 * n_k * (n_k + 1) // 2
    # E_x alone through Parseval: the three forward products per block
    plan.profile(True)
    e_only = kx.kx_energy_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ)).item()
    prof = plan.profile_read()
    assert prof["bloch"][1] == 3 * n_k * (n_k + 1) // 2
    assert abs(e_only - ex_ref) < TOL_K[prec][1] * abs(ex_ref)


@pytest.mark.parametrize("case", [8, 9, 10, 11])
def test_kpoint_tensor_core_and_cuda_core_products(kx, case, monkeypatch):
    """Axes of 32 and 64 points run their products on the tensor cores (split
    fp16, per-tile scale); with KX_BLOCH_TC=0 the same plan uses the CUDA-core
    kernels.  Both match the oracle; chunks of 5 pairs make tiles straddle
    items."""
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(case, 340 + case)
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel)
    vx_ref, ex_ref = oracle.vx_kpoints(base, theta, wk, psi, occ)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    monkeypatch.setenv("KX_CHUNK_PAIRS", "5")
    out = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("KX_BLOCH_TC", tc)
        vx, ex = kx.kx_vx_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ))
        e_only = kx.kx_energy_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ)).item()
        torch.cuda.synchronize()
        assert plan.status() == kx.KX_OK
        vx = vx.cpu().numpy().transpose(0, 2, 1)
        assert relmax(vx, vx_ref) < TOL_K[prec][0], tc
        assert abs(ex.item() - ex_ref) < TOL_K[prec][1] * abs(ex_ref), tc
        assert abs(e_only - ex_ref) < TOL_K[prec][1] * abs(ex_ref), tc
        out[tc] = vx
    assert relmax(out["1"], out["0"]) < TOL_K[prec][0]


@pytest.mark.parametrize("case", [12, 13])
def test_kpoint_pass_kernels_and_tile_kernels(kx, case, monkeypatch):
    """With every axis of 32 or 64 points the products run in the pass kernels
    (split scales per item: a bound from the orbital maxima for the first ones,
    then the maxima the previous product recorded); KX_BLOCH_PASS=0 takes the
    per-tile-maximum kernels instead.  Both match the oracle, with whole chunks
    and with chunks of 5 pairs, and E_x alone agrees."""
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(case, 360 + case)
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel)
    vx_ref, ex_ref = oracle.vx_kpoints(base, theta, wk, psi, occ)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    out = {}
    for chunk in (None, "5"):
        if chunk:
            monkeypatch.setenv("KX_CHUNK_PAIRS", chunk)
        for bp in ("1", "0"):
            monkeypatch.setenv("KX_BLOCH_PASS", bp)
            vx, ex = kx.kx_vx_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ))
            e_only = kx.kx_energy_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ)).item()
            torch.cuda.synchronize()
            assert plan.status() == kx.KX_OK
            vx = vx.cpu().numpy().transpose(0, 2, 1)
            assert relmax(vx, vx_ref) < TOL_K[prec][0], (chunk, bp)
            assert abs(ex.item() - ex_ref) < TOL_K[prec][1] * abs(ex_ref), (chunk, bp)
            assert abs(e_only - ex_ref) < TOL_K[prec][1] * abs(ex_ref), (chunk, bp)
            out[(chunk, bp)] = vx
    assert relmax(out[(None, "1")], out[(None, "0")]) < TOL_K[prec][0]
    assert relmax(out[("5", "1")], out[(None, "1")]) < TOL_K[prec][0]


@pytest.mark.parametrize("prec", [0, 1])
def test_kpoint_apply_to_vectors_in_chunks(kx, prec, monkeypatch):
    """Vx at one k-point on arbitrary complex vectors, with chunks of 4 pairs that
    split a vector's bands across chunks, and without occupations."""
    sysd, theta, wk, psi, _, _ = kpoint_inputs(1, 311)
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((sysd.N, 5)) + 1j * rng.standard_normal((sysd.N, 5))
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel)
    ref = oracle.vx_apply_kpoint(base, theta, wk, psi, None, 2, phi)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    monkeypatch.setenv("KX_CHUNK_PAIRS", "4")
    plan.profile(True)
    out = kx.kx_vx_apply_kpoint(plan, theta, wk, to_dev_orbitals(psi), 2, dev(phi.T))
    torch.cuda.synchronize()
    prof = plan.profile_read()
    assert prof["bloch"][1] == 6 * len(wk) * 4  # 15 pairs per q in chunks of 4
    assert relmax(out.cpu().numpy().T, ref) < TOL_K[prec][0]
    # the energy alone in chunks of 4 of the 9 pairs per block (chunks that
    # split a k-point's bands), with occupations
    occ = np.random.default_rng(6).uniform(0.2, 1.0, (len(wk), psi.shape[2]))
    e_ref = oracle.exchange_energy_kpoints(base, theta, wk, psi, occ)
    e = kx.kx_energy_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ)).item()
    assert abs(e - e_ref) < TOL_K[prec][1] * abs(e_ref)


def test_kpoint_gamma_with_real_orbitals_is_the_real_path(kx):
    n, h, bc, kind = (12, 10, 14), (0.45, 0.5, 0.4), (P, P, D), U
    sysd = system(n, h, bc, kind, 4, 321)
    psi = workloads.make_orbitals(sysd)
    occ = np.array([1.0, 0.9, 0.5, 0.2])
    plan = kx.Plan(n, h, bc, kind, precision=0)
    vx_r, ex_r = kx.kx_vx_apply(plan, dev(psi.T), dev(occ))
    vx_c, ex_c = kx.kx_vx_kpoints(plan, [[0.0, 0.0, 0.0]], [1.0], dev(psi.T.astype(np.complex128)[None]),
                                  dev(occ[None]))
    vx_c = vx_c.cpu().numpy()[0]
    assert relmax(vx_c.real, vx_r.cpu().numpy()) < 1e-11
    assert np.max(np.abs(vx_c.imag)) < 1e-11 * np.max(np.abs(vx_c.real))
    assert abs(ex_c.item() - ex_r.item()) < 1e-11 * abs(ex_r.item())


def test_kpoint_rejects_bad_arguments(kx):
    import ctypes
    sysd, theta, wk, psi, occ, _ = kpoint_inputs(0, 330)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=0)
    psi_d = to_dev_orbitals(psi)
    phi = psi_d[1].clone()
    for bad_k in (-1, len(wk)):
        with pytest.raises(kx.KxError) as ei:
            kx.kx_vx_apply_kpoint(plan, theta, wk, psi_d, bad_k, phi)
        assert ei.value.code == kx.KX_ERR_ARG
    th_bad = theta.copy()
    th_bad[1, 0] = np.nan
    with pytest.raises(kx.KxError) as ei:
        kx.kx_vx_kpoints(plan, th_bad, wk, psi_d)
    assert ei.value.code == kx.KX_ERR_ARG
    with pytest.raises(kx.KxError) as ei:
        kx.kx_vx_apply_kpoint(plan, theta, wk, psi_d, 0, phi, out=psi_d[0])
    assert ei.value.code == kx.KX_ERR_ARG
    # a complex buffer that starts 8 bytes into an allocation
    raw = torch.zeros(2 * plan.N * 3 + 2, dtype=torch.float64, device="cuda")
    ta = (ctypes.c_double * (3 * len(wk)))(*theta.ravel())
    wa = (ctypes.c_double * len(wk))(*wk)
    rc = kx.lib().kx_vx_apply_kpoint(plan.handle, len(wk), ctypes.cast(ta, ctypes.c_void_p),
                                     ctypes.cast(wa, ctypes.c_void_p), psi.shape[2],
                                     ctypes.c_void_p(psi_d.data_ptr()), None, 0, 1,
                                     ctypes.c_void_p(raw.data_ptr() + 8), ctypes.c_void_p(phi.data_ptr()),
                                     kx._stream())
    assert rc == kx.KX_ERR_ARG
    mp = kx.Plan((16, 16, 16), (0.5,) * 3, (D, D, D), U, precision=0)
    mp.set_multipole(2)
    x = torch.zeros((1, 1, mp.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(kx.KxError) as ei:
        kx.kx_vx_kpoints(mp, [[0.0, 0.0, 0.0]], [1.0], x)
    assert ei.value.code == kx.KX_ERR_UNSUPPORTED
    assert plan.status() == kx.KX_OK


def test_kpoint_full_size_sampled(kx):
    """The 64^3 slab with 16 bands on a 2 x 2 k-grid (the k-point workload the
    benchmark times): two runs are bit-identical, one band's Vx at one k-point
    matches the oracle, and E_x matches its definition from the returned Vx."""
    sysd = workloads.K1
    theta, wk = workloads.kpoint_grid(sysd, workloads.K1_KGRID)
    psi = workloads.make_bloch_orbitals(sysd, theta)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=1)
    psi_d = to_dev_orbitals(psi)
    vx, ex = kx.kx_vx_kpoints(plan, theta, wk, psi_d)
    vx2, ex2 = kx.kx_vx_kpoints(plan, theta, wk, psi_d)
    torch.cuda.synchronize()
    assert torch.equal(vx, vx2) and ex.item() == ex2.item()  # deterministic
    base = oracle.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel)
    k, band = 1, 5
    ref = oracle.vx_apply_kpoint(base, theta, wk, psi, None, k, psi[k][:, band:band + 1])[:, 0]
    got = vx[k, band].cpu().numpy()
    assert relmax(got, ref) < TOL_K[1][0]
    vxn = vx.cpu().numpy()
    e_def = 0.5 * sysd.dV * sum(wk[q] * np.vdot(psi[q][:, m], vxn[q, m]).real
                               for q in range(len(wk)) for m in range(sysd.n_orb))
    assert abs(ex.item() - e_def) < 1e-9 * abs(e_def) and ex.item() < 0


# ---------------------------------------------------------------- invariances (no oracle)
@pytest.mark.parametrize("prec", [0, 1])
def test_invariances_on_gpu(kx, prec):
    """Orbital rotation (E_x fixed, Vx psi -> (Vx psi) U), axis permutation (the
    transposed grid gives the transposed result) and scaling (Vx(c psi) =
    c^3 Vx(psi), E_x(c psi) = c^4 E_x(psi)) through the CUDA path."""
    n, h, bc, kind = (16, 24, 32), (0.45, 0.4, 0.5), (D, P, D), S
    sysd = system(n, h, bc, kind, 5, 401)
    psi = workloads.make_orbitals(sysd)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    vx0, ex0 = kx.kx_vx_apply(plan, dev(psi.T))
    vx0 = vx0.cpu().numpy().T
    ex0 = ex0.item()
    tv, te = TOL[prec]["vx"], TOL[prec]["ex"]
    # rotation
    U, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((5, 5)))
    vxr, exr = kx.kx_vx_apply(plan, dev((psi @ U).T))
    assert relmax(vxr.cpu().numpy().T, vx0 @ U) < 10 * tv
    assert abs(exr.item() - ex0) < 10 * te * abs(ex0)
    # axis permutation x1 <-> x2
    n_p, h_p, bc_p = (n[1], n[0], n[2]), (h[1], h[0], h[2]), (bc[1], bc[0], bc[2])
    cube = psi.reshape(n[2], n[1], n[0], 5)
    psi_p = np.ascontiguousarray(cube.transpose(0, 2, 1, 3)).reshape(-1, 5)
    plan_p = kx.Plan(n_p, h_p, bc_p, kind, precision=prec)
    vxp, exp_ = kx.kx_vx_apply(plan_p, dev(psi_p.T))
    ref_p = vx0.reshape(n[2], n[1], n[0], 5).transpose(0, 2, 1, 3).reshape(-1, 5)
    assert relmax(vxp.cpu().numpy().T, ref_p) < 10 * tv
    assert abs(exp_.item() - ex0) < 10 * te * abs(ex0)
    # scaling
    c = 1.7
    vxs, exs = kx.kx_vx_apply(plan, dev((c * psi).T))
    assert relmax(vxs.cpu().numpy().T, c ** 3 * vx0) < 10 * tv
    assert abs(exs.item() - c ** 4 * ex0) < 10 * te * abs(c ** 4 * ex0)


@pytest.mark.parametrize("case", [1, 9])
def test_kpoint_gauge_invariance(kx, case):
    """A global phase per k-point on the Bloch orbitals (a gauge change) leaves
    E_x unchanged and multiplies Vx psi_k by the same phase."""
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(case, 420 + case)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    vx0, ex0 = kx.kx_vx_kpoints(plan, theta, wk, to_dev_orbitals(psi), dev(occ))
    vx0 = vx0.cpu().numpy()
    alpha = np.random.default_rng(11).uniform(0, 2 * np.pi, len(wk))
    ph = np.exp(1j * alpha)
    vx1, ex1 = kx.kx_vx_kpoints(plan, theta, wk, to_dev_orbitals(psi * ph[:, None, None]), dev(occ))
    assert relmax(vx1.cpu().numpy(), vx0 * ph[:, None, None]) < 5 * TOL_K[prec][0]
    assert abs(ex1.item() - ex0.item()) < 5 * TOL_K[prec][1] * abs(ex0.item())


@pytest.mark.parametrize("case", [0, 1])
def test_kpoint_block_ranges_sum_to_full(kx, case):
    """kx_vx_kpoint_blocks over the ranges a multi-GPU split would give each rank
    (shard.kpoint_block_range) adds up to kx_vx_kpoints; an empty range gives
    zeros; a range past the last block is rejected."""
    from paper_2406_16998_gb300 import shard
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(case, 450 + case)
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    psi_d, occ_d = to_dev_orbitals(psi), dev(occ)
    full, ef = kx.kx_vx_kpoints(plan, theta, wk, psi_d, occ_d)
    full = full.cpu().numpy()
    acc, e = np.zeros_like(full), 0.0
    for rank in range(3):
        a, b = shard.kpoint_block_range(len(wk), rank, 3)
        part, ep = kx.kx_vx_kpoint_blocks(plan, theta, wk, psi_d, a, b, occ_d)
        acc += part.cpu().numpy()
        e += ep.item()
    assert relmax(acc, full) < 1e-12
    assert abs(e - ef.item()) < 1e-12 * abs(ef.item())
    zero, ez = kx.kx_vx_kpoint_blocks(plan, theta, wk, psi_d, 2, 2, occ_d)
    assert zero.abs().max().item() == 0.0 and ez.item() == 0.0
    B = len(wk) * (len(wk) + 1) // 2
    with pytest.raises(kx.KxError) as ei:
        kx.kx_vx_kpoint_blocks(plan, theta, wk, psi_d, 0, B + 1, occ_d)
    assert ei.value.code == kx.KX_ERR_ARG


def test_kpoint_empty_block_range_on_a_fresh_plan(kx):
    """The share of a rank that gets no k-point block (one k-point split over two
    ranks: rank 0 owns [0, 0)) as the very first call on a new plan, with E_x
    requested: zeros, E_x = 0, no error, status clean; the other rank's share
    then equals kx_vx_kpoints."""
    from paper_2406_16998_gb300 import shard
    sysd, theta, wk, psi, occ, prec = kpoint_inputs(1, 470)
    theta, wk, psi, occ = theta[:1], np.ones(1), psi[:1], occ[:1]
    psi_d, occ_d = to_dev_orbitals(psi), dev(occ)
    ranges = [shard.kpoint_block_range(1, r, 2) for r in range(2)]
    assert ranges == [(0, 0), (0, 1)]
    plan = kx.Plan(sysd.n, sysd.h, sysd.bc, sysd.kernel, precision=prec)
    zero, ez = kx.kx_vx_kpoint_blocks(plan, theta, wk, psi_d, *ranges[0], occ_d)
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK
    assert zero.abs().max().item() == 0.0 and ez.item() == 0.0
    part, ep = kx.kx_vx_kpoint_blocks(plan, theta, wk, psi_d, *ranges[1], occ_d)
    full, ef = kx.kx_vx_kpoints(plan, theta, wk, psi_d, occ_d)
    assert relmax(part.cpu().numpy(), full.cpu().numpy()) < 1e-12
    assert abs(ep.item() - ef.item()) < 1e-12 * abs(ef.item())


# --------------------------------------------------------------------------
# Config 5 as configured: E_x of the 80^3 periodic screened 256-orbital system
# through the autograd function, split-precision forward, float64 sums.
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c5(kx):
    sysd = workloads.C5
    psi = dev(workloads.make_orbitals(sysd).T)                      # (256, N)
    plan = kx.Plan.for_system(sysd, precision=1)
    x = psi.clone().requires_grad_(True)
    E = kx.exchange_energy(x, plan)
    E.backward()
    plan64 = kx.Plan.for_system(sysd, precision=0)
    g64, e64 = kx.kx_energy_gradient(plan64, psi)
    torch.cuda.synchronize()
    assert plan.status() == kx.KX_OK and plan64.status() == kx.KX_OK
    return dict(sysd=sysd, psi=psi, grad=x.grad.detach(), e=E.item(), g64=g64, e64=e64.item(), plan64=plan64)


def test_c5_gradient_against_fp64_plan(kx, c5):
    """The backward of the split-precision autograd function (2 dV g Vx psi,
    pair products recomputed) against the float64 plan's gradient on the whole
    80^3 x 256 output, and the forward E_x (Parseval) against the float64 plan's."""
    g, g64 = c5["grad"], c5["g64"]
    assert float((g - g64).abs().max() / g64.abs().max()) < TOL[1]["vx"]
    assert abs(c5["e"] - c5["e64"]) < TOL[1]["ex"] * abs(c5["e64"])


def test_c5_central_differences(kx, c5):
    """Central differences (step 1e-4) of the float64 E_x at 16 random
    (orbital, grid point) entries of the 80^3 / 256-orbital system, against the
    float64 gradient and the split-precision autograd gradient.  Only the pair
    solves that involve the perturbed orbital change E_x, so the orbital is
    moved to the front of the set and E_x is taken over the block pairs of
    orbital block 0 with every block (kx_vx_apply_block_pairs: orbitals 0..3
    with every orbital, 1018 pairs), which hold all of them; the other pairs
    cancel in the difference.  About 32 float64 solves of 1018 pairs (~20 s of
    GPU time)."""
    from paper_2406_16998_gb300 import shard
    sysd, psi, plan64 = c5["sysd"], c5["psi"], c5["plan64"]
    n_orb, N = psi.shape
    row0 = [(0, J) for J in range(shard.n_blocks(n_orb))]
    assert len(shard.pairs_of_block_pairs(n_orb, row0)) == 1018
    rng = np.random.default_rng(5)
    step = 1e-4
    gmax64 = c5["g64"].abs().max().item()
    gmax = c5["grad"].abs().max().item()
    out = torch.empty_like(psi)
    ep = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(16):
        k, r = int(rng.integers(n_orb)), int(rng.integers(N))
        perm = torch.tensor([k] + [o for o in range(n_orb) if o != k], device="cuda")
        p = psi.index_select(0, perm).contiguous()
        v0 = p[0, r].item()
        e = []
        for d in (step, -step):
            p[0, r] = v0 + d
            kx.kx_vx_apply_block_pairs(plan64, p, row0, out=out, e_x=ep)
            e.append(ep.item())
        fd = (e[0] - e[1]) / (2 * step)
        assert abs(fd - c5["g64"][k, r].item()) < 1e-6 * gmax64
        assert abs(fd - c5["grad"][k, r].item()) < TOL[1]["vx"] * gmax
    assert plan64.status() == kx.KX_OK


@pytest.mark.parametrize("prec", [0, 1])
def test_block_pair_shares_match_oracle_and_sum_to_full(kx, prec):
    """kx_vx_apply_block_pairs over the 2D block-cyclic shares of four ranks:
    each share against the oracle's sums over its pairs, the shares summing to
    kx_vx_apply; an empty share gives zeros; a repeated or out-of-range block
    pair is rejected."""
    from paper_2406_16998_gb300 import shard
    n, h, bc, kind = (24, 40, 16), (0.45, 0.4, 0.5), (D, P, D), S
    sysd = system(n, h, bc, kind, 11, 480)
    psi = workloads.make_orbitals(sysd)
    op = oracle.Plan(n, h, bc, kind)
    plan = kx.Plan(n, h, bc, kind, precision=prec)
    psi_d = dev(psi.T)
    full, ef = kx.kx_vx_apply(plan, psi_d)
    acc, e = torch.zeros_like(full), 0.0
    world = 4
    for r in range(world):
        bps = shard.rank_block_pairs(sysd.n_orb, r, world)
        part, ep = kx.kx_vx_apply_block_pairs(plan, psi_d, bps)
        ref, e_ref = oracle.vx_apply(op, psi, pairs=shard.pairs_of_block_pairs(sysd.n_orb, bps))
        assert relmax(part.cpu().numpy().T, ref) < TOL[prec]["vx"]
        assert abs(ep.item() - e_ref) < TOL[prec]["ex"] * abs(e_ref)
        acc += part
        e += ep.item()
    assert relmax(acc.cpu().numpy(), full.cpu().numpy()) < (1e-12 if prec == 0 else 1e-6)
    assert abs(e - ef.item()) < (1e-12 if prec == 0 else 1e-7) * abs(ef.item())
    zero, ez = kx.kx_vx_apply_block_pairs(plan, psi_d, [])
    assert zero.abs().max().item() == 0.0 and ez.item() == 0.0
    for bad in ([(0, 1), (0, 1)], [(1, 0)], [(0, 3)]):
        with pytest.raises(kx.KxError) as ei:
            kx.kx_vx_apply_block_pairs(plan, psi_d, bad)
        assert ei.value.code == kx.KX_ERR_ARG
    assert plan.status() == kx.KX_OK


def test_c4_batch_of_the_eight_systems_against_oracle(kx):
    """Config 4 as configured: the eight systems of uneven grids, boundary
    conditions and kernels (16-128 orbitals) in one batch graph, each plan tuned
    by kx_batch_create.  For every system, orbital 0's row of Vx psi (its pair
    solves with every orbital) against the oracle, E_x against
    1/2 dV sum_i <psi_i, (Vx psi)_i>, and a second run bit-identical to the first."""
    plans, psis, outs = [], [], []
    for sd in workloads.C4:
        plans.append(kx.Plan.for_system(sd, precision=1))
        psis.append(dev(workloads.make_orbitals(sd).T))
        outs.append(torch.empty_like(psis[-1]))
    batch = kx.Batch(plans, [sd.n_orb for sd in workloads.C4])
    exs = torch.empty(len(plans), dtype=torch.float64, device="cuda")
    batch.run(psis, outs, e_x=exs)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    batch.run(psis, outs, e_x=exs)
    torch.cuda.synchronize()
    for k, sd in enumerate(workloads.C4):
        assert plans[k].status() == kx.KX_OK
        assert plans[k].tuning()["tuned_ms"] > 0.0
        assert torch.equal(first[k], outs[k])
        psi_h = psis[k].cpu().numpy()
        vxh = outs[k].cpu().numpy()
        e_id = 0.5 * sd.dV * float(np.einsum("ij,ij->", psi_h, vxh))
        assert abs(exs[k].item() - e_id) < 1e-6 * abs(e_id)
        op = oracle.Plan(sd.n, sd.h, sd.bc, sd.kernel, sd.omega, sd.fd_order)
        ref, _ = oracle.vx_apply(op, psi_h.T, ordered=True, pairs=[(0, j) for j in range(sd.n_orb)])
        assert np.max(np.abs(vxh[0] - ref[:, 0])) < TOL[1]["vx"] * np.abs(ref[:, 0]).max(), sd.name
    batch.close()


@pytest.mark.parametrize("n_orb", [1, 5, 9, 30])
def test_host_path_pieces_and_ragged_blocks(kx, n_orb, monkeypatch):
    """kx_vx_apply_host with the orbitals sent in pieces for sizes that leave a
    ragged last orbital block, a single block (every group holds the last
    block) and more pieces than the first two chunk cuts: Vx psi bit for bit
    the device path's, E_x to the last bits, both against the oracle; with
    occupations."""
    monkeypatch.setenv("KX_CHUNK_PAIRS", "24")
    n, h, bc = (16, 24, 32), (0.45, 0.4, 0.5), (D, D, P)
    sysd = system(n, h, bc, S, n_orb, 500 + n_orb)
    psi = workloads.make_orbitals(sysd)
    occ = np.random.default_rng(n_orb).uniform(0.3, 1.0, n_orb)
    op = oracle.Plan(n, h, bc, S)
    vx_ref, ex_ref = oracle.vx_apply(op, psi, occ=occ)
    plan = kx.Plan(n, h, bc, S, precision=1)
    vx, ex = kx.kx_vx_apply(plan, dev(psi.T), occ=dev(occ))
    vx_h, ex_h = kx.kx_vx_apply_host(plan, torch.from_numpy(np.ascontiguousarray(psi.T)).pin_memory(),
                                     occ_host=torch.from_numpy(occ))
    assert plan.status() == kx.KX_OK
    assert np.array_equal(vx_h.numpy(), vx.cpu().numpy())
    assert abs(ex_h - ex.item()) <= 1e-13 * abs(ex.item())
    assert relmax(vx_h.numpy().T, vx_ref) < TOL[1]["vx"]
    assert abs(ex_h - ex_ref) < TOL[1]["ex"] * abs(ex_ref)
