"""GPU test of kx_apply_fL_noalloc, the entry point for callers that cannot
allocate device memory at the point of the call: their device memory was
reserved up front (a pool or caching allocator owns it), or they run inside a
solver loop where a cudaMalloc / cudaFree, with its device-wide
synchronisation, is not allowed.

The entry point must give what the FP64 oracle and kx_apply_fL give, call after
call, and the device's free memory must not change while it runs, also on a
plan whose own workspace has never been sized (so that growing a plan-owned
buffer would show).  Collected last on purpose (file name), so that a run
stopping at the first failure has already run every other test.  It passes run
alone in a fresh process and after the other tests."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F16X3 = 1e-5  # the split-precision tolerance used by the other parity tests
GRID = ((24, 40, 16), (0.45, 0.4, 0.5), (0, 1, 0), 1)  # n, h, bc (D, P, D), screened


@pytest.fixture(scope="module")
def kx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2406_16998_gb300 import build
    build.build()
    import paper_2406_16998_gb300 as k
    return k


def _relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_matches_oracle_on_a_fresh_plan_without_allocating(kx):
    n, h, bc, kind = GRID
    b1_h = workloads.random_field(n[0] * n[1] * n[2], 3, 5)          # (N, 3)
    b2_h = workloads.random_field(n[0] * n[1] * n[2], 5, 6) * 1e-3   # different size and scale
    op = oracle.Plan(n, h, bc, kind)
    ref1, ref2 = oracle.apply_fL(op, b1_h).T, oracle.apply_fL(op, b2_h).T
    b1 = torch.from_numpy(np.ascontiguousarray(b1_h.T)).cuda()
    b2 = torch.from_numpy(np.ascontiguousarray(b2_h.T)).cuda()
    out1, out2, out3 = torch.empty_like(b1), torch.empty_like(b2), torch.empty_like(b1)

    # warm-up on another plan of the same grid: the first call on the device may
    # load the library's tensor-core code and the static array, and each kernel
    # of the path is loaded at its first launch
    warm = kx.Plan(n, h, bc, kind, precision=kx.KX_F16X3)
    kx.kx_apply_fL_noalloc(warm, b1, out3)
    torch.cuda.synchronize()

    # a fresh plan: its workspace has never been sized
    plan = kx.Plan(n, h, bc, kind, precision=kx.KX_F16X3)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    kx.kx_apply_fL_noalloc(plan, b1, out1)      # two calls in a row
    kx.kx_apply_fL_noalloc(plan, b2, out2)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    assert plan.status() == kx.KX_OK

    assert _relmax(out1.cpu().numpy(), ref1) < TOL_F16X3
    assert _relmax(out2.cpu().numpy(), ref2) < TOL_F16X3
    # the allocating entry point agrees within the same tolerance
    assert _relmax(out1.cpu().numpy(), kx.kx_apply_fL(plan, b1).cpu().numpy()) < TOL_F16X3
    # a third call with the first input again: no state carried over from call two
    kx.kx_apply_fL_noalloc(plan, b1, out3)
    torch.cuda.synchronize()
    assert _relmax(out3.cpu().numpy(), ref1) < TOL_F16X3


def test_noalloc_rejects_requests_beyond_its_scratch(kx):
    n, h, bc, kind = (24, 40, 16), (0.45, 0.4, 0.5), (0, 0, 0), 0
    plan = kx.Plan(n, h, bc, kind, precision=kx.KX_F16X3)
    n_rhs = 2_621_440 // plan.N + 1
    b = torch.zeros((n_rhs, plan.N), dtype=torch.float64, device="cuda")
    out = torch.empty_like(b)
    with pytest.raises(kx.KxError) as ei:
        kx.kx_apply_fL_noalloc(plan, b, out)
    assert ei.value.code == kx.KX_ERR_ARG
    assert "exceeds the static scratch limit" in str(ei.value)
