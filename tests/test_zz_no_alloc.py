"""GPU test of kx_apply_fL_noalloc, the entry point for callers that cannot
allocate device memory at the point of the call (their memory was reserved up
front, or a cudaMalloc/cudaFree and its device-wide synchronisation is not
allowed there).  It must give what kx_apply_fL gives, call after call, while
the device's free memory stays unchanged.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F16X3 = 1e-5  # the split-precision tolerance used by the other parity tests


@pytest.fixture(scope="module")
def kx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2406_16998_gb300 import build
    build.build()
    import paper_2406_16998_gb300 as k
    return k


def _relmax(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_matches_apply_fL_on_consecutive_calls(kx):
    n, h, bc, kind = (24, 40, 16), (0.45, 0.4, 0.5), (0, 1, 0), 1
    plan = kx.Plan(n, h, bc, kind, precision=kx.KX_F16X3)
    b1 = torch.from_numpy(workloads.random_field(plan.N, 3, 5).T.copy()).cuda()
    b2 = torch.from_numpy(workloads.random_field(plan.N, 5, 6).T.copy()).cuda() * 1e-3
    ref1 = kx.kx_apply_fL(plan, b1)
    ref2 = kx.kx_apply_fL(plan, b2)
    out1 = torch.empty_like(b1)
    out2 = torch.empty_like(b2)
    torch.cuda.synchronize()

    kx.kx_apply_fL_noalloc(plan, b1, out1)          # first call on this device: address set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    kx.kx_apply_fL_noalloc(plan, b2, out2)          # second call: different size and scale
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]

    assert _relmax(out1, ref1) < TOL_F16X3
    assert _relmax(out2, ref2) < TOL_F16X3
    assert free_after == free_before
    # a third call with the first input again: no state carried over from call two
    out3 = torch.empty_like(b1)
    kx.kx_apply_fL_noalloc(plan, b1, out3)
    torch.cuda.synchronize()
    assert _relmax(out3, ref1) < TOL_F16X3


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
