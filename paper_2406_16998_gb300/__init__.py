"""Python binding of the kronx C-ABI library (libkronx.so).

Argument marshalling only: every step of the exchange apply runs in the CUDA
kernels of the library.  Importing this module does not need a GPU; the first
call that needs the library loads it and raises if it has not been built.
PyTorch provides device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkronx.so")

KX_DIRICHLET, KX_PERIODIC = 0, 1
KX_UNSCREENED, KX_SCREENED = 0, 1
KX_FP64, KX_F16X3, KX_FFT32 = 0, 1, 2
KX_OK, KX_ERR_ARG, KX_ERR_SINGULAR, KX_ERR_NOMEM, KX_ERR_CUDA, KX_ERR_TIMEOUT, KX_ERR_UNSUPPORTED = range(7)

# Every symbol the C header declares, with (restype, argtypes).
_c_int, _c_double, _vp, _ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong


class KxGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("bc", ctypes.c_int * 3),
                ("fd_order", ctypes.c_int)]


class KxKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("omega", ctypes.c_double)]


SIGNATURES = {
    "kx_plan_create": (_c_int, [ctypes.POINTER(KxGrid), ctypes.POINTER(KxKernel), _c_int, ctypes.POINTER(_vp)]),
    "kx_plan_destroy": (_c_int, [_vp]),
    "kx_plan_eig": (_c_int, [_vp, _c_int, _vp, _vp]),
    "kx_plan_ftable": (_c_int, [_vp, _vp]),
    "kx_apply_fL": (_c_int, [_vp, _c_int, _vp, _vp, _vp]),
    "kx_apply_fL_noalloc": (_c_int, [_vp, _c_int, _vp, _vp, _vp]),
    "kx_vx_apply": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "kx_vx_apply_host": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "kx_vx_apply_pairs": (_c_int, [_vp, _c_int, _vp, _vp, _ll, _ll, _vp, _vp, _vp]),
    "kx_vx_apply_block_pairs": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _c_int, _vp, _vp, _vp]),
    "kx_energy": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp]),
    "kx_ace": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "kx_ace_apply": (_c_int, [_vp, _c_int, _vp, _c_int, _vp, _vp, _vp]),
    "kx_plan_set_multipole": (_c_int, [_vp, _c_int]),
    "kx_vx_apply_kpoint": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _c_int, _c_int, _vp, _vp, _vp]),
    "kx_vx_kpoints": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "kx_energy_kpoints": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp, _vp]),
    "kx_vx_kpoint_blocks": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _ll, _ll, _vp, _vp, _vp]),
    "kx_energy_gradient": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "kx_batch_create": (_c_int, [_c_int, _vp, _vp, ctypes.POINTER(_vp)]),
    "kx_batch_run": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "kx_batch_destroy": (_c_int, [_vp]),
    "kx_autotune": (_c_int, [_vp, _c_int, _c_int]),
    "kx_plan_tuning": (_c_int, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                ctypes.POINTER(ctypes.c_float)]),
    "kx_plan_status": (_c_int, [_vp, ctypes.POINTER(_c_int), _vp]),
    "kx_selftest_wait": (_c_int, [_vp, _ll, _vp]),
    "kx_profile": (_c_int, [_vp, _c_int]),
    "kx_profile_read": (_c_int, [_vp, _c_int, _vp, _vp]),
    "kx_last_error_detail": (_c_int, [ctypes.c_char_p, _c_int]),
    "kx_strerror": (ctypes.c_char_p, [_c_int]),
}

_lib = None


def lib():
    """Load libkronx.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2406_16998_gb300.build.build() "
                               "(the exchange apply has no CPU or PyTorch fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class KxError(RuntimeError):
    def __init__(self, code, detail):
        self.code = code
        name = lib().kx_strerror(code).decode()
        super().__init__(f"{name}: {detail}")


def _check(rc):
    if rc != KX_OK:
        buf = ctypes.create_string_buffer(512)
        lib().kx_last_error_detail(buf, 512)
        raise KxError(rc, buf.value.decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, name, dtype=None, shape=None):
    torch = _torch()
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """One grid + kernel + precision (kx_plan_create / kx_plan_destroy)."""

    def __init__(self, n, h, bc, kind, omega=0.11, fd_order=12, precision=KX_F16X3):
        g = KxGrid()
        for a in range(3):
            g.n[a] = int(n[a])
            g.h[a] = float(h[a])
            g.bc[a] = int(bc[a])
        g.fd_order = int(fd_order)
        k = KxKernel(int(kind), float(omega))
        handle = ctypes.c_void_p()
        self._h = None
        _check(lib().kx_plan_create(ctypes.byref(g), ctypes.byref(k), int(precision), ctypes.byref(handle)))
        self._h = handle
        self.n = tuple(int(x) for x in n)
        self.h = tuple(float(x) for x in h)
        self.bc = tuple(int(x) for x in bc)
        self.kind = int(kind)
        self.omega = float(omega)
        self.fd_order = int(fd_order)
        self.precision = int(precision)

    @classmethod
    def for_system(cls, sysd, precision=KX_F16X3):
        return cls(sysd.n, sysd.h, sysd.bc, sysd.kernel, sysd.omega, sysd.fd_order, precision)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    @property
    def N(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def dV(self):
        return self.h[0] * self.h[1] * self.h[2]

    def close(self):
        if self._h is not None:
            lib().kx_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_multipole(self, l_max: int):
        """Dirichlet values from the multipole expansion of each source up to
        order l_max (-1: zero boundary values); see kx_plan_set_multipole."""
        _check(lib().kx_plan_set_multipole(self.handle, int(l_max)))
        self.l_max = int(l_max)

    def eig(self, axis):
        n = self.n[axis]
        lam = np.empty(n)
        V = np.empty((n, n))
        _check(lib().kx_plan_eig(self.handle, axis, lam.ctypes.data_as(_vp), V.ctypes.data_as(_vp)))
        return lam, V

    def ftable(self):
        f = np.empty(self.N)
        _check(lib().kx_plan_ftable(self.handle, f.ctypes.data_as(_vp)))
        return f

    PROFILE_KINDS = ["prep", "X3F", "X2F", "X1", "X2I", "X3I", "final", "fp64_mode", "fp64_other", "ace",
                     "setup", "acc", "slab", "ace_comb", "multipole", "fft", "bloch",
                     "bloch_other"]

    def profile(self, enable=True):
        _check(lib().kx_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """{kind: (total_ms, launches)} since the last profile() call."""
        k = len(self.PROFILE_KINDS)
        ms = np.zeros(k)
        ln = np.zeros(k, dtype=np.int64)
        _check(lib().kx_profile_read(self.handle, k, ms.ctypes.data_as(_vp), ln.ctypes.data_as(_vp)))
        return {name: (float(ms[i]), int(ln[i])) for i, name in enumerate(self.PROFILE_KINDS)}

    def tuning(self):
        """{chunk_pairs, fuse_slab, pass_stages, tuned_ms} of the plan's launch shapes (kx_plan_tuning)."""
        ch, fz, st, ms = _ll(0), _c_int(0), _c_int(0), ctypes.c_float(0.0)
        _check(lib().kx_plan_tuning(self.handle, ctypes.byref(ch), ctypes.byref(fz), ctypes.byref(st),
                                    ctypes.byref(ms)))
        return {"chunk_pairs": ch.value, "fuse_slab": fz.value, "pass_stages": st.value, "tuned_ms": ms.value}

    def status(self, stream=None):
        st = ctypes.c_int(0)
        _check(lib().kx_plan_status(self.handle, ctypes.byref(st), _stream(stream)))
        return st.value


def kx_apply_fL(plan: Plan, b, out=None, stream=None):
    """X = f(L) B for b of shape (n_rhs, N), float64 CUDA tensor."""
    torch = _torch()
    n_rhs = b.shape[0]
    if out is None:
        out = torch.empty_like(b)
    _check(lib().kx_apply_fL(plan.handle, n_rhs, _dptr(b, "b", torch.float64, (n_rhs, plan.N)),
                             _dptr(out, "out", torch.float64, (n_rhs, plan.N)), _stream(stream)))
    return out


def kx_apply_fL_noalloc(plan: Plan, b, out, stream=None):
    """X = f(L) B through the allocation-free entry point (scratch is a static
    array inside the library).  `out` must be supplied by the caller, so the
    call allocates nothing on the device; see kronx.h for the size limit."""
    torch = _torch()
    n_rhs = b.shape[0]
    _check(lib().kx_apply_fL_noalloc(plan.handle, n_rhs, _dptr(b, "b", torch.float64, (n_rhs, plan.N)),
                                     _dptr(out, "out", torch.float64, (n_rhs, plan.N)), _stream(stream)))
    return out


def kx_vx_apply(plan: Plan, psi, occ=None, out=None, e_x=None, stream=None):
    """(Vx psi, E_x) for psi of shape (n_orb, N), float64 CUDA tensor; E_x is a 1-element tensor."""
    torch = _torch()
    n_orb = psi.shape[0]
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(lib().kx_vx_apply(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)),
                             _dptr(occ, "occ", torch.float64, (n_orb,)),
                             _dptr(out, "out", torch.float64, (n_orb, plan.N)),
                             _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_vx_apply_pairs(plan: Plan, psi, pair_begin, pair_end, occ=None, out=None, e_x=None, stream=None):
    """Partial (Vx psi, E_x) over pairs [pair_begin, pair_end) of the symmetric list."""
    torch = _torch()
    n_orb = psi.shape[0]
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(lib().kx_vx_apply_pairs(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)),
                                   _dptr(occ, "occ", torch.float64, (n_orb,)), int(pair_begin), int(pair_end),
                                   _dptr(out, "out", torch.float64, (n_orb, plan.N)),
                                   _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_vx_apply_block_pairs(plan: Plan, psi, blocks, occ=None, out=None, e_x=None, stream=None):
    """Partial (Vx psi, E_x) over the orbital block pairs `blocks` (a sequence of
    (I, J), I <= J, blocks of four orbitals); see kx_vx_apply_block_pairs."""
    torch = _torch()
    n_orb = psi.shape[0]
    flat = [int(x) for bp in blocks for x in bp]
    arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(lib().kx_vx_apply_block_pairs(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)),
                                         _dptr(occ, "occ", torch.float64, (n_orb,)), ctypes.cast(arr, _vp),
                                         len(flat) // 2, _dptr(out, "out", torch.float64, (n_orb, plan.N)),
                                         _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_energy(plan: Plan, psi, occ=None, e_x=None, stream=None):
    torch = _torch()
    n_orb = psi.shape[0]
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(lib().kx_energy(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)),
                           _dptr(occ, "occ", torch.float64, (n_orb,)),
                           _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return e_x


def kx_vx_apply_host(plan: Plan, psi_host, occ_host=None, out=None, stream=None):
    """Host-buffer variant: psi_host is a CPU float64 tensor (pinned recommended); returns (vx, E_x)."""
    torch = _torch()
    n_orb = psi_host.shape[0]
    if psi_host.is_cuda or psi_host.dtype != torch.float64 or not psi_host.is_contiguous():
        raise TypeError("psi_host must be a contiguous CPU float64 tensor")
    if out is None:
        out = torch.empty_like(psi_host, pin_memory=psi_host.is_pinned())
    ex = np.zeros(1)
    occ_p = None
    if occ_host is not None:
        occ_p = ctypes.c_void_p(occ_host.data_ptr())
    _check(lib().kx_vx_apply_host(plan.handle, n_orb, ctypes.c_void_p(psi_host.data_ptr()), occ_p,
                                  ctypes.c_void_p(out.data_ptr()), ex.ctypes.data_as(_vp), _stream(stream)))
    return out, float(ex[0])


def kx_ace(plan: Plan, psi, vx_psi, stream=None):
    """(xi, M) of the compressed exchange operator built from psi and vx_psi."""
    torch = _torch()
    n_orb = psi.shape[0]
    xi = torch.empty_like(psi)
    M = torch.empty((n_orb, n_orb), dtype=torch.float64, device=psi.device)
    _check(lib().kx_ace(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)),
                        _dptr(vx_psi, "vx_psi", torch.float64, (n_orb, plan.N)), _dptr(xi, "xi"),
                        _dptr(M, "M"), _stream(stream)))
    return xi, M


def kx_energy_gradient(plan: Plan, psi, occ=None, out=None, e_x=None, stream=None):
    """(dE_x/dpsi, E_x): 2 dV g_a G_a, G = Vx psi (symmetric form of the multipole
    correction when the plan has one); see kx_energy_gradient in kronx.h."""
    torch = _torch()
    n_orb = psi.shape[0]
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    occ_p = None if occ is None else _dptr(occ, "occ", torch.float64, (n_orb,))
    _check(lib().kx_energy_gradient(plan.handle, n_orb, _dptr(psi, "psi", torch.float64, (n_orb, plan.N)), occ_p,
                                    _dptr(out, "out", torch.float64, (n_orb, plan.N)),
                                    _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_ace_apply(plan: Plan, xi, phi, out=None, stream=None):
    """V_ACE phi = -xi (dV xi^T phi) for the n_vec grid vectors phi (rows of a float64 tensor)."""
    torch = _torch()
    n_xi, n_vec = xi.shape[0], phi.shape[0]
    if out is None:
        out = torch.empty_like(phi)
    _check(lib().kx_ace_apply(plan.handle, n_xi, _dptr(xi, "xi", torch.float64, (n_xi, plan.N)), n_vec,
                              _dptr(phi, "phi", torch.float64, (n_vec, plan.N)),
                              _dptr(out, "out", torch.float64, (n_vec, plan.N)), _stream(stream)))
    return out


def _kpoint_host(theta, wk):
    th = [float(x) for row in theta for x in row]
    w = [float(x) for x in wk]
    if len(th) != 3 * len(w):
        raise ValueError("theta must hold 3 phases per k-point")
    ta = (ctypes.c_double * len(th))(*th)
    wa = (ctypes.c_double * len(w))(*w)
    return len(w), ta, wa


def kx_vx_apply_kpoint(plan: Plan, theta, wk, psi, k_index: int, phi, occ=None, out=None, stream=None):
    """Vx at k-point k_index applied to complex vectors phi (n_vec x N, complex128),
    with the orbitals psi (n_kpt x n_orb x N, complex128) at the k-points whose
    phases per cell are theta (n_kpt x 3) and weights wk; see kx_vx_apply_kpoint."""
    torch = _torch()
    n_kpt, ta, wa = _kpoint_host(theta, wk)
    n_orb, n_vec = psi.shape[1], phi.shape[0]
    if out is None:
        out = torch.empty_like(phi)
    occ_p = None if occ is None else _dptr(occ, "occ", torch.float64, (n_kpt, n_orb))
    _check(lib().kx_vx_apply_kpoint(plan.handle, n_kpt, ctypes.cast(ta, _vp), ctypes.cast(wa, _vp), n_orb,
                                    _dptr(psi, "psi", torch.complex128, (n_kpt, n_orb, plan.N)), occ_p,
                                    int(k_index), n_vec, _dptr(phi, "phi", torch.complex128, (n_vec, plan.N)),
                                    _dptr(out, "out", torch.complex128, (n_vec, plan.N)), _stream(stream)))
    return out


def kx_vx_kpoints(plan: Plan, theta, wk, psi, occ=None, out=None, e_x=None, stream=None):
    """(Vx psi at every k-point, E_x) for complex128 orbitals psi (n_kpt x n_orb x N);
    see kx_vx_kpoints."""
    torch = _torch()
    n_kpt, ta, wa = _kpoint_host(theta, wk)
    n_orb = psi.shape[1]
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    occ_p = None if occ is None else _dptr(occ, "occ", torch.float64, (n_kpt, n_orb))
    _check(lib().kx_vx_kpoints(plan.handle, n_kpt, ctypes.cast(ta, _vp), ctypes.cast(wa, _vp), n_orb,
                               _dptr(psi, "psi", torch.complex128, (n_kpt, n_orb, plan.N)), occ_p,
                               _dptr(out, "vx", torch.complex128, (n_kpt, n_orb, plan.N)),
                               _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_vx_kpoint_blocks(plan: Plan, theta, wk, psi, block_begin: int, block_end: int, occ=None, out=None, e_x=None,
                        stream=None):
    """Partial (Vx psi at every k-point, E_x) from the k-point blocks
    [block_begin, block_end) (see kx_vx_kpoint_blocks and shard.kpoint_blocks)."""
    torch = _torch()
    n_kpt, ta, wa = _kpoint_host(theta, wk)
    n_orb = psi.shape[1]
    if out is None:
        out = torch.empty_like(psi)
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    occ_p = None if occ is None else _dptr(occ, "occ", torch.float64, (n_kpt, n_orb))
    _check(lib().kx_vx_kpoint_blocks(plan.handle, n_kpt, ctypes.cast(ta, _vp), ctypes.cast(wa, _vp), n_orb,
                                     _dptr(psi, "psi", torch.complex128, (n_kpt, n_orb, plan.N)), occ_p,
                                     int(block_begin), int(block_end),
                                     _dptr(out, "vx", torch.complex128, (n_kpt, n_orb, plan.N)),
                                     _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return out, e_x


def kx_energy_kpoints(plan: Plan, theta, wk, psi, occ=None, e_x=None, stream=None):
    """E_x alone for complex128 orbitals psi (n_kpt x n_orb x N); see kx_energy_kpoints."""
    torch = _torch()
    n_kpt, ta, wa = _kpoint_host(theta, wk)
    n_orb = psi.shape[1]
    if e_x is None:
        e_x = torch.empty(1, dtype=torch.float64, device=psi.device)
    occ_p = None if occ is None else _dptr(occ, "occ", torch.float64, (n_kpt, n_orb))
    _check(lib().kx_energy_kpoints(plan.handle, n_kpt, ctypes.cast(ta, _vp), ctypes.cast(wa, _vp), n_orb,
                                   _dptr(psi, "psi", torch.complex128, (n_kpt, n_orb, plan.N)), occ_p,
                                   _dptr(e_x, "e_x", torch.float64, (1,)), _stream(stream)))
    return e_x


def kx_autotune(plan: Plan, n_orb: int, budget_ms: int = 2000):
    _check(lib().kx_autotune(plan.handle, int(n_orb), int(budget_ms)))


def kx_selftest_wait(plan: Plan, max_cycles: int, stream=None):
    _check(lib().kx_selftest_wait(plan.handle, int(max_cycles), _stream(stream)))


class Batch:
    """Several systems' exchange applies in one CUDA graph (kx_batch_create / run / destroy)."""

    def __init__(self, plans, n_orb):
        self.plans = list(plans)
        self.n_orb = [int(x) for x in n_orb]
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        norb = (ctypes.c_int * len(self.plans))(*self.n_orb)
        h = ctypes.c_void_p()
        self._h = None
        _check(lib().kx_batch_create(len(self.plans), arr, norb, ctypes.byref(h)))
        self._h = h

    def run(self, psis, outs, e_x=None, stream=None):
        torch = _torch()
        n = len(self.plans)
        for k in range(n):
            _dptr(psis[k], "psi", torch.float64, (self.n_orb[k], self.plans[k].N))
            _dptr(outs[k], "out", torch.float64, (self.n_orb[k], self.plans[k].N))
        pa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in psis])
        oa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
        _check(lib().kx_batch_run(self._h, pa, oa, _dptr(e_x, "e_x", torch.float64, (n,)), _stream(stream)))

    def close(self):
        if self._h is not None:
            lib().kx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    torch = _torch()

    class ExchangeEnergy(torch.autograd.Function):
        """E_x(psi) with a hand-written backward: dE_x/dpsi_k = 2 dV g_k G_k,
        G = Vx psi (with the symmetric form of the multipole correction when the
        plan has one).

        forward runs kx_energy (forward transforms and the Parseval sum only);
        backward recomputes the pair products inside kx_energy_gradient (nothing
        stored).
        """

        @staticmethod
        def forward(ctx, psi, plan, occ=None):
            ctx.plan = plan
            ctx.save_for_backward(psi, occ) if occ is not None else ctx.save_for_backward(psi)
            ctx.has_occ = occ is not None
            return kx_energy(plan, psi.detach().contiguous(), occ)[0].clone()

        @staticmethod
        def backward(ctx, g_e):
            saved = ctx.saved_tensors
            psi = saved[0]
            occ = saved[1] if ctx.has_occ else None
            grad, _ = kx_energy_gradient(ctx.plan, psi.detach().contiguous(), occ)
            return grad * g_e, None, None

    return ExchangeEnergy


def exchange_energy(psi, plan: Plan, occ=None):
    """Differentiable E_x (torch.autograd)."""
    return _autograd().apply(psi, plan, occ)
