"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function named ``lbm_*`` here forwards to the CUDA library entry point of
the same name; all lattice arithmetic runs in the library's kernels. PyTorch is
used only for device memory (output tensors) and for the CUDA stream. The
library must have been built (``paper_2009_04352_gb300.build.build()``); if it
is missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

Q = 19
K_STATS = 11
K_WALL = 4

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_ERR_DIVERGED = -4
LBM_ERR_STATE = -5

WALL_BB, WALL_WFB, WALL_FREESLIP, WALL_WFB_NODE = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_CELL, KERNEL_PAIR, KERNEL_TMA, KERNEL_QUAD = 0, 1, 2, 3, 4
COLLISION_BGK, COLLISION_MRT = 0, 1
LAW_SPALDING, LAW_LOG, LAW_POWER = 0, 1, 2
FP32, FP16_SHIFTED = 0, 1
PULL2, AA = 0, 1
BATCH_PERSISTENT, BATCH_MEMBER_GRIDS = 1, 2


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class lbm_wall_model(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa", C.c_double), ("B", C.c_double), ("y1", C.c_double),
                ("nu", C.c_double), ("newton_iters", C.c_int), ("law", C.c_int)]


class lbm_member(C.Structure):
    _fields_ = [("grid", lbm_grid), ("tau", C.c_double), ("C_s", C.c_double), ("force", C.c_double * 3),
                ("wall", lbm_wall_model)]


_lock = threading.Lock()
_lib = None

_DP = C.POINTER(C.c_double)
_FP = C.POINTER(C.c_float)
_VP = C.c_void_p

_SIGNATURES = {
    "lbm_create": (C.c_int, [lbm_grid, C.c_double, C.c_double, _DP, lbm_wall_model, C.c_int, C.c_int,
                             _VP, C.POINTER(_VP)]),
    "lbm_population_bytes": (C.c_size_t, [lbm_grid, C.c_int]),
    "lbm_create_from_buffers": (C.c_int, [lbm_grid, C.c_double, C.c_double, _DP, lbm_wall_model, C.c_int,
                                          C.c_int, _VP, _VP, _VP, C.POINTER(_VP)]),
    "lbm_init_channel": (C.c_int, [_VP, _DP, C.c_double, C.c_uint64]),
    "lbm_set_populations": (C.c_int, [_VP, _DP]),
    "lbm_populations": (C.c_int, [_VP, _DP]),
    "lbm_set_stats_every": (C.c_int, [_VP, C.c_int]),
    "lbm_step": (C.c_int, [_VP, C.c_int]),
    "lbm_get_step": (C.c_longlong, [_VP]),
    "lbm_set_kernel": (C.c_int, [_VP, C.c_int]),
    "lbm_get_kernel": (C.c_int, [_VP]),
    "lbm_autotune": (C.c_int, [_VP, C.c_int, _DP, C.POINTER(C.c_int)]),
    "lbm_set_les": (C.c_int, [_VP, C.c_int, C.c_double, C.c_double]),
    "lbm_moments": (C.c_int, [_VP, _VP, _VP, C.c_int]),
    "lbm_wall_stress": (C.c_int, [_VP, _VP, C.c_int]),
    "lbm_plane_stats": (C.c_int, [_VP, _DP, _DP, C.POINTER(C.c_longlong), C.c_int]),
    "lbm_conservation": (C.c_int, [_VP, _DP]),
    "lbm_plane_profile_noalloc": (C.c_int, [_VP, _VP]),
    "lbm_sync": (C.c_int, [_VP]),
    "lbm_set_wait_limit": (C.c_int, [_VP, C.c_longlong]),
    "lbm_batch_create": (C.c_int, [C.c_int, C.POINTER(lbm_member), C.c_int, _VP, C.POINTER(_VP)]),
    "lbm_batch_member": (_VP, [_VP, C.c_int]),
    "lbm_batch_cells": (C.c_longlong, [_VP]),
    "lbm_batch_set_stats_every": (C.c_int, [_VP, C.c_int]),
    "lbm_batch_step": (C.c_int, [_VP, C.c_int]),
    "lbm_batch_set_config": (C.c_int, [_VP, C.c_int, C.c_int]),
    "lbm_batch_get_config": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_longlong)]),
    "lbm_batch_set_form": (C.c_int, [_VP, C.c_int, C.c_int]),
    "lbm_batch_get_form": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "lbm_batch_autotune": (C.c_int, [_VP, C.c_int, _DP]),
    "lbm_batch_set_les": (C.c_int, [_VP, C.c_int, _DP, C.c_double]),
    "lbm_batch_sync": (C.c_int, [_VP]),
    "lbm_batch_destroy": (None, [_VP]),
    "lbm_destroy": (None, [_VP]),
    "lbm_last_error": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
            h = C.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
        return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(rc):
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm_last_error().decode())
    return rc


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------ raw entry points

def lbm_create(nx, ny, nz, tau, cs, force, wall=WALL_WFB, kappa=0.41, B=5.5, y1=1.0, nu=-1.0,
               newton_iters=12, precision=FP32, layout=PULL2, stream=None, law=LAW_SPALDING):
    g = lbm_grid(int(nx), int(ny), int(nz))
    wm = lbm_wall_model(int(wall), float(kappa), float(B), float(y1), float(nu), int(newton_iters), int(law))
    fvec = np.ascontiguousarray(np.asarray(force, dtype=np.float64).reshape(3))
    out = C.c_void_p()
    s = _current_stream() if stream is None else C.c_void_p(stream)
    _check(lib().lbm_create(g, float(tau), float(cs), _dp(fvec), wm, int(precision), int(layout), s,
                            C.byref(out)))
    return out


def lbm_population_bytes(nx, ny, nz, precision=FP32):
    return int(lib().lbm_population_bytes(lbm_grid(int(nx), int(ny), int(nz)), int(precision)))


def lbm_create_from_buffers(nx, ny, nz, tau, cs, force, pop0, pop1, wall=WALL_WFB, kappa=0.41, B=5.5, y1=1.0,
                            nu=-1.0, newton_iters=12, precision=FP32, layout=PULL2, stream=None, law=LAW_SPALDING):
    """pop0, pop1: device addresses (ints) of caller-owned population arrays."""
    g = lbm_grid(int(nx), int(ny), int(nz))
    wm = lbm_wall_model(int(wall), float(kappa), float(B), float(y1), float(nu), int(newton_iters), int(law))
    fvec = np.ascontiguousarray(np.asarray(force, dtype=np.float64).reshape(3))
    out = C.c_void_p()
    s = _current_stream() if stream is None else C.c_void_p(stream)
    _check(lib().lbm_create_from_buffers(g, float(tau), float(cs), _dp(fvec), wm, int(precision), int(layout), s,
                                         C.c_void_p(pop0), C.c_void_p(pop1), C.byref(out)))
    return out


def lbm_init_channel(h, u_mean_x, noise_amp, seed):
    um = np.ascontiguousarray(np.asarray(u_mean_x, dtype=np.float64))
    _check(lib().lbm_init_channel(h, _dp(um), float(noise_amp), C.c_uint64(int(seed))))


def lbm_set_populations(h, f: np.ndarray):
    _check(lib().lbm_set_populations(h, _dp(np.ascontiguousarray(f, dtype=np.float64))))


def lbm_populations(h, out: np.ndarray):
    _check(lib().lbm_populations(h, _dp(out)))
    return out


def lbm_set_stats_every(h, every):
    _check(lib().lbm_set_stats_every(h, int(every)))


def lbm_step(h, n):
    _check(lib().lbm_step(h, int(n)))


def lbm_get_step(h):
    return int(lib().lbm_get_step(h))


def lbm_set_kernel(h, kernel):
    _check(lib().lbm_set_kernel(h, int(kernel)))


def lbm_get_kernel(h):
    return int(lib().lbm_get_kernel(h))


def lbm_autotune(h, steps):
    """Time every kernel form the grid allows and keep the fastest; returns
    (kernel, ms per step)."""
    ms, k = C.c_double(), C.c_int()
    _check(lib().lbm_autotune(h, int(steps), C.byref(ms), C.byref(k)))
    return int(k.value), float(ms.value)


def lbm_set_les(h, collision, u_tau_ref=0.0, a_plus=0.0):
    _check(lib().lbm_set_les(h, int(collision), float(u_tau_ref), float(a_plus)))


def lbm_moments(h, rho_ptr, u_ptr, on_device):
    _check(lib().lbm_moments(h, C.c_void_p(rho_ptr), C.c_void_p(u_ptr), int(on_device)))


def lbm_wall_stress(h, ptr, on_device):
    _check(lib().lbm_wall_stress(h, C.c_void_p(ptr), int(on_device)))


def lbm_plane_stats(h, out, wall_out, reset):
    ns = C.c_longlong(0)
    _check(lib().lbm_plane_stats(h, _dp(out) if out is not None else None,
                                 _dp(wall_out) if wall_out is not None else None, C.byref(ns),
                                 int(bool(reset))))
    return ns.value


def lbm_conservation(h, out):
    rc = lib().lbm_conservation(h, _dp(out))
    _check(rc)
    return out


def lbm_plane_profile_noalloc(h, out_dev_ptr):
    _check(lib().lbm_plane_profile_noalloc(h, C.c_void_p(out_dev_ptr)))


def lbm_sync(h):
    _check(lib().lbm_sync(h))


def lbm_set_wait_limit(h, cycles):
    _check(lib().lbm_set_wait_limit(h, int(cycles)))


def lbm_destroy(h):
    lib().lbm_destroy(h)


# ------------------------------------------------------------ convenience class

class Channel:
    """One channel lattice on the current CUDA device (wraps an lbm_handle)."""

    def __init__(self, nx, ny, nz, tau, cs, force, wall=WALL_WFB, kappa=0.41, B=5.5, y1=1.0, nu=-1.0,
                 newton_iters=12, precision=FP32, layout=PULL2, stream=None, law=LAW_SPALDING):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self.precision, self.layout, self.wall, self.collision = precision, layout, wall, COLLISION_BGK
        self._h = lbm_create(nx, ny, nz, tau, cs, force, wall, kappa, B, y1, nu, newton_iters, precision,
                             layout, stream, law)

    @classmethod
    def from_buffers(cls, case, buffers, precision=FP32, wall=None, stream=None, layout=PULL2):
        """A channel whose population arrays are caller-owned device tensors
        (one for AA, two for the two-lattice layout), each of at least
        lbm_population_bytes bytes; the channel keeps them referenced."""
        self = cls.__new__(cls)
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        self.n = self.nx * self.ny * self.nz
        self.precision, self.layout, self.collision = precision, layout, COLLISION_BGK
        self.wall = case.wall if wall is None else wall
        need = lbm_population_bytes(case.nx, case.ny, case.nz, precision)
        for t in buffers:
            if not t.is_cuda or t.numel() * t.element_size() < need:
                raise ValueError(f"each population buffer must be a CUDA tensor of >= {need} bytes")
        ptrs = [t.data_ptr() for t in buffers] + [None] * (2 - len(buffers))
        self._buffers = tuple(buffers)
        self._h = lbm_create_from_buffers(case.nx, case.ny, case.nz, case.tau, case.cs, case.force, ptrs[0], ptrs[1],
                                          case.wall if wall is None else wall, case.kappa, case.b_const, case.y1,
                                          case.nu_wall, case.newton_iters, precision, layout, stream, case.wall_law)
        return self

    @classmethod
    def from_case(cls, case, precision=FP32, wall=None, stream=None, layout=PULL2):
        return cls(case.nx, case.ny, case.nz, case.tau, case.cs, case.force,
                   case.wall if wall is None else wall, case.kappa, case.b_const, case.y1,
                   case.nu_wall, case.newton_iters, precision, layout, stream, case.wall_law)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_channel(self, u_mean_x, noise_amp, seed):
        lbm_init_channel(self._h, u_mean_x, noise_amp, seed)

    def set_populations(self, f):
        lbm_set_populations(self._h, np.asarray(f, dtype=np.float64).reshape(Q, -1))

    def populations(self):
        out = np.zeros((Q, self.nz, self.ny, self.nx))
        return lbm_populations(self._h, out)

    def set_stats_every(self, every):
        lbm_set_stats_every(self._h, every)

    def step(self, n=1):
        lbm_step(self._h, n)

    @property
    def step_count(self):
        return lbm_get_step(self._h)

    @property
    def kernel(self):
        return lbm_get_kernel(self._h)

    def set_kernel(self, kernel):
        lbm_set_kernel(self._h, kernel)

    def autotune(self, steps=16):
        """Select the fastest kernel form for this grid (advances the state by
        steps + 2 per form tried). Returns (kernel, ms per step)."""
        return lbm_autotune(self._h, steps)

    def set_les(self, collision=COLLISION_BGK, u_tau_ref=0.0, a_plus=0.0):
        lbm_set_les(self._h, collision, u_tau_ref, a_plus)
        self.collision = collision

    def moments(self, device=False):
        """(rho [nz,ny,nx], u [3,nz,ny,nx]) as FP32 numpy arrays, or torch CUDA
        tensors when device=True."""
        if device:
            import torch
            rho = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float32, device="cuda")
            u = torch.empty((3, self.nz, self.ny, self.nx), dtype=torch.float32, device="cuda")
            lbm_moments(self._h, rho.data_ptr(), u.data_ptr(), 1)
            return rho, u
        rho = np.zeros((self.nz, self.ny, self.nx), dtype=np.float32)
        u = np.zeros((3, self.nz, self.ny, self.nx), dtype=np.float32)
        lbm_moments(self._h, rho.ctypes.data, u.ctypes.data, 0)
        return rho, u

    def wall_stress(self):
        out = np.zeros((2, self.nz, self.nx, 2), dtype=np.float32)
        lbm_wall_stress(self._h, out.ctypes.data, 0)
        return out

    def plane_stats(self, reset=False):
        out = np.zeros((self.ny, K_STATS))
        w = np.zeros((2, K_WALL))
        ns = lbm_plane_stats(self._h, out, w, reset)
        return out, w, ns

    def conservation(self):
        return lbm_conservation(self._h, np.zeros(4))

    def sync(self):
        lbm_sync(self._h)

    def set_wait_limit(self, cycles):
        lbm_set_wait_limit(self._h, cycles)


# ------------------------------------------------------------ batched ensemble

def member_of(case):
    m = lbm_member()
    m.grid = lbm_grid(case.nx, case.ny, case.nz)
    m.tau = case.tau
    m.C_s = case.cs
    for i in range(3):
        m.force[i] = case.force[i]
    m.wall = lbm_wall_model(case.wall, case.kappa, case.b_const, case.y1, case.nu_wall, case.newton_iters,
                            case.wall_law)
    return m


class _MemberView(Channel):
    """A batch member seen through the single-channel API (owned by the batch)."""

    def __init__(self, handle, case, precision):
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        self.n = self.nx * self.ny * self.nz
        self.precision = precision
        self._h = handle

    def close(self):
        self._h = None


class Batch:
    """Ensemble of independent channels advanced by one launch per step."""

    def __init__(self, cases, precision=FP32, stream=None):
        arr = (lbm_member * len(cases))(*[member_of(c) for c in cases])
        out = C.c_void_p()
        s = _current_stream() if stream is None else C.c_void_p(stream)
        _check(lib().lbm_batch_create(len(cases), arr, int(precision), s, C.byref(out)))
        self._b = out
        self.cases = list(cases)
        self.precision = precision
        self.members = [_MemberView(C.c_void_p(lib().lbm_batch_member(out, i)), c, precision)
                        for i, c in enumerate(cases)]

    @property
    def handle(self):
        return self._b

    @property
    def cells(self):
        return int(lib().lbm_batch_cells(self._b))

    def set_stats_every(self, every):
        _check(lib().lbm_batch_set_stats_every(self._b, int(every)))

    def step(self, n=1):
        _check(lib().lbm_batch_step(self._b, int(n)))

    def set_config(self, threads, ctas_per_sm):
        _check(lib().lbm_batch_set_config(self._b, int(threads), int(ctas_per_sm)))

    def config(self):
        t, c, g, tl = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
        _check(lib().lbm_batch_get_config(self._b, C.byref(t), C.byref(c), C.byref(g), C.byref(tl)))
        st = C.c_int()
        form = int(lib().lbm_batch_get_form(self._b, C.byref(st)))
        return {"threads": t.value, "ctas_per_sm": c.value, "grid": g.value, "tiles": tl.value,
                "form": form, "streams": st.value}

    def set_form(self, form, streams=0):
        _check(lib().lbm_batch_set_form(self._b, int(form), int(streams)))

    @property
    def form(self):
        return int(lib().lbm_batch_get_form(self._b, None))

    def set_les(self, collision=COLLISION_BGK, u_tau_ref=None, a_plus=0.0):
        ut = None if u_tau_ref is None else np.ascontiguousarray(np.asarray(u_tau_ref, dtype=np.float64))
        _check(lib().lbm_batch_set_les(self._b, int(collision), _dp(ut) if ut is not None else None,
                                       float(a_plus)))

    def autotune(self, steps=5):
        ms = C.c_double()
        _check(lib().lbm_batch_autotune(self._b, int(steps), C.byref(ms)))
        return ms.value

    def sync(self):
        _check(lib().lbm_batch_sync(self._b))

    def close(self):
        if self._b:
            for m in self.members:
                m.close()
            lib().lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
