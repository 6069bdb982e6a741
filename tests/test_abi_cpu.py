"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a,
loads, exports every function include/kronx.h declares, and rejects bad
arguments before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "kronx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kx_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def kx():
    from paper_2406_16998_gb300 import build
    build.build()
    import paper_2406_16998_gb300 as k
    return k


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["kx_plan_create", "kx_plan_destroy", "kx_vx_apply", "kx_energy", "kx_apply_fL", "kx_ace",
                     "kx_ace_apply", "kx_vx_apply_kpoint", "kx_vx_kpoints", "kx_vx_kpoint_blocks", "kx_energy_kpoints", "kx_batch_create",
                     "kx_batch_run", "kx_autotune", "kx_last_error_detail", "kx_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(kx):
    L = kx.lib()
    for name in header_functions():
        assert hasattr(L, name), f"{name} declared in kronx.h but not exported"
    # the binding knows every declared function, with a signature
    assert set(header_functions()) == set(kx.SIGNATURES)


def test_strerror_names(kx):
    L = kx.lib()
    assert L.kx_strerror(0) == b"KX_OK"
    assert L.kx_strerror(2) == b"KX_ERR_SINGULAR"
    assert L.kx_strerror(5) == b"KX_ERR_TIMEOUT"
    assert L.kx_strerror(99) == b"KX_ERR_UNKNOWN"


def _create(kx, n, h, bc, fd, kind, omega, prec):
    g = kx.KxGrid()
    for a in range(3):
        g.n[a], g.h[a], g.bc[a] = n[a], h[a], bc[a]
    g.fd_order = fd
    k = kx.KxKernel(kind, omega)
    out = ctypes.c_void_p()
    rc = kx.lib().kx_plan_create(ctypes.byref(g), ctypes.byref(k), prec, ctypes.byref(out))
    buf = ctypes.create_string_buffer(256)
    kx.lib().kx_last_error_detail(buf, 256)
    return rc, buf.value.decode()


@pytest.mark.parametrize("args,code", [
    (((1, 8, 8), (0.5,) * 3, (0, 0, 0), 12, 0, 0.11, 0), 1),        # n < 2
    (((8, 8, 200), (0.5,) * 3, (0, 0, 0), 12, 0, 0.11, 0), 6),      # n > 128
    (((8, 8, 8), (0.5, 0.0, 0.5), (0, 0, 0), 12, 0, 0.11, 0), 1),   # h <= 0
    (((8, 8, 8), (0.5,) * 3, (0, 2, 0), 12, 0, 0.11, 0), 1),        # bad bc
    (((8, 8, 8), (0.5,) * 3, (0, 0, 0), 11, 0, 0.11, 0), 1),        # odd order
    (((8, 8, 8), (0.5,) * 3, (0, 0, 0), 12, 1, 0.0, 0), 1),         # screened, omega 0
    (((8, 8, 8), (0.5,) * 3, (0, 0, 0), 12, 0, 0.11, 7), 1),        # bad precision
    (((8, 12, 8), (0.5,) * 3, (0, 0, 0), 12, 0, 0.11, 1), 6),       # F16X3 needs n % 8 == 0
    (((8, 8, 8), (0.5,) * 3, (1, 1, 1), 12, 0, 0.11, 0), 2),        # singular
])
def test_plan_create_rejects_bad_arguments(kx, args, code):
    rc, msg = _create(kx, *args)
    assert rc == code, msg
    assert msg


def test_null_arguments(kx):
    L = kx.lib()
    assert L.kx_plan_create(None, None, 0, None) == 1
    assert L.kx_vx_apply(None, 1, None, None, None, None, None) == 1
    assert L.kx_apply_fL(None, 1, None, None, None) == 1
    assert L.kx_plan_destroy(None) == 0
    assert L.kx_batch_destroy(None) == 0
    # the k-point calls reject a missing plan before any argument is used
    assert L.kx_vx_kpoints(None, 1, None, None, 1, None, None, None, None, None) == 1
    assert L.kx_vx_apply_kpoint(None, 1, None, None, 1, None, None, 0, 1, None, None, None) == 1
    assert L.kx_energy_kpoints(None, 1, None, None, 1, None, None, None, None) == 1
