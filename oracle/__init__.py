"""FP64 CPU oracle of the WFB LBM-LES channel update (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this module; the library under
``paper_2009_04352_gb300`` never does. It shares no code with the CUDA path.

Every function here is a thin ctypes call into ``lbm_oracle.c``; the arithmetic
lives there, written in plain double precision as the paper's equations read
(Eqs. 1-2 and 14-17, Sec. 2-3). Where the paper is silent or garbled (the
corrected populations of Eq. 14c, the wall distance of Eq. 17, the forcing
scheme, the Smagorinsky closure) the function concerned states the reading it
takes in its comment.

Parity status: every oracle function has at least one independent pin in
``tests/test_oracle_pins.py``; none is marked "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
K_STATS = 11


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction, no fast-math;
    OpenMP for the all-cores timing mode where the compiler has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
        if subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:] + ["-lm"], capture_output=True).returncode != 0:
            subprocess.run(base + ["-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        vp = C.c_void_p
        sig = {
            "or_table": (None, [ip, dp, ip, ip]),
            "or_feq": (None, [C.c_double, dp, dp]),
            "or_moments_cell": (None, [dp, dp, dp, dp]),
            "or_pi_neq": (None, [dp, dp, dp]),
            "or_tau_eff": (C.c_double, [C.c_double, C.c_double, C.c_double, dp]),
            "or_guo": (None, [C.c_double, dp, dp, dp]),
            "or_collide": (None, [dp, C.c_double, C.c_double, dp, dp, dp, dp, dp]),
            "or_spalding_yplus": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "or_spalding_newton": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int,
                                             C.c_double, dp, dp]),
            "or_wfb_stress": (None, [C.c_double, dp, C.c_double, C.c_double, C.c_double,
                                     C.c_double, dp]),
            "or_wfb_stress_law": (None, [C.c_int, C.c_double, dp, C.c_double, C.c_double,
                                         C.c_double, C.c_double, dp]),
            "or_loglaw_crossing": (C.c_double, [C.c_double, C.c_double]),
            "or_loglaw_uplus": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "or_powerlaw_uplus": (C.c_double, [C.c_double]),
            "or_wall_uplus": (C.c_double, [C.c_int, C.c_double, C.c_double, C.c_double]),
            "or_set_wall_law": (C.c_int, [vp, C.c_int]),
            "or_splitmix64": (C.c_uint64, [C.c_uint64]),
            "or_uniform": (C.c_double, [C.c_uint64, C.c_uint64]),
            "or_create": (vp, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp, C.c_int,
                               C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]),
            "or_destroy": (None, [vp]),
            "or_init_channel": (None, [vp, dp, C.c_double, C.c_uint64]),
            "or_set_populations": (None, [vp, dp]),
            "or_get_populations": (None, [vp, dp]),
            "or_moments": (None, [vp, dp, dp]),
            "or_conservation": (None, [vp, dp]),
            "or_wall_stress": (None, [vp, dp]),
            "or_wall_delta_f": (None, [vp, dp]),
            "or_plane_stats": (None, [vp, dp, dp, C.POINTER(C.c_longlong), C.c_int]),
            "or_get_step": (C.c_longlong, [vp]),
            "or_step": (None, [vp, C.c_int]),
            "or_mrt_matrix": (None, [dp]),
            "or_mrt_rates": (None, [C.c_double, dp]),
            "or_collide_mrt": (None, [dp, C.c_double, C.c_double, dp, C.c_double, dp, dp, dp, dp]),
            "or_collide_mrt_rates": (None, [dp, C.c_double, C.c_double, dp, C.c_double, dp, dp, dp, dp, dp]),
            "or_van_driest": (C.c_double, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
            "or_set_les": (None, [vp, C.c_int, C.c_double, C.c_double]),
            "or_set_threads": (C.c_int, [vp, C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ------------------------------------------------------------ cell level --

def table():
    """D3Q19 velocities e[19,3], weights w[19], opposite[19], y-mirror[19]."""
    lib = _load()
    e = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    mir = np.zeros(19, dtype=np.int32)
    ip = C.POINTER(C.c_int)
    lib.or_table(e.ctypes.data_as(ip), _dp(w), opp.ctypes.data_as(ip), mir.ctypes.data_as(ip))
    return e.reshape(19, 3), w, opp, mir


def feq(rho, u):
    out = np.zeros(19)
    _load().or_feq(float(rho), _dp(_vec(u, 3)), _dp(out))
    return out


def moments_cell(f, F):
    rho = np.zeros(1)
    u = np.zeros(3)
    _load().or_moments_cell(_dp(_vec(f, 19)), _dp(_vec(F, 3)), _dp(rho), _dp(u))
    return rho[0], u


def pi_neq(f, fe):
    out = np.zeros(9)
    _load().or_pi_neq(_dp(_vec(f, 19)), _dp(_vec(fe, 19)), _dp(out))
    return out.reshape(3, 3)


def tau_eff(tau0, cs, rho, pi):
    return _load().or_tau_eff(float(tau0), float(cs), float(rho), _dp(_vec(pi, 9)))


def guo(tau, u, F):
    out = np.zeros(19)
    _load().or_guo(float(tau), _dp(_vec(u, 3)), _dp(_vec(F, 3)), _dp(out))
    return out


def collide(f, tau0, cs, F):
    """Returns (f*, rho, u, tau_eff) for one cell."""
    fs = np.zeros(19)
    rho = np.zeros(1)
    u = np.zeros(3)
    tau = np.zeros(1)
    _load().or_collide(_dp(_vec(f, 19)), float(tau0), float(cs), _dp(_vec(F, 3)), _dp(fs),
                       _dp(rho), _dp(u), _dp(tau))
    return fs, rho[0], u, tau[0]


def mrt_matrix():
    out = np.zeros(19 * 19)
    _load().or_mrt_matrix(_dp(out))
    return out.reshape(19, 19)


def mrt_rates(tau):
    out = np.zeros(19)
    _load().or_mrt_rates(float(tau), _dp(out))
    return out


def collide_mrt(f, tau0, cs, F, damp=1.0):
    """Returns (f*, rho, u, tau_eff) for one cell with the MRT operator."""
    fs = np.zeros(19)
    rho = np.zeros(1)
    u = np.zeros(3)
    tau = np.zeros(1)
    _load().or_collide_mrt(_dp(_vec(f, 19)), float(tau0), float(cs), _dp(_vec(F, 3)), float(damp), _dp(fs),
                           _dp(rho), _dp(u), _dp(tau))
    return fs, rho[0], u, tau[0]


def collide_mrt_rates(f, tau0, cs, F, rates, damp=1.0):
    fs = np.zeros(19)
    rho = np.zeros(1)
    u = np.zeros(3)
    tau = np.zeros(1)
    _load().or_collide_mrt_rates(_dp(_vec(f, 19)), float(tau0), float(cs), _dp(_vec(F, 3)), float(damp),
                                 _dp(_vec(rates, 19)), _dp(fs), _dp(rho), _dp(u), _dp(tau))
    return fs, rho[0], u, tau[0]


def van_driest(j, ny, u_tau, nu, a_plus=26.0):
    return _load().or_van_driest(int(j), int(ny), float(u_tau), float(nu), float(a_plus))


def spalding_yplus(up, kappa=0.41, B=5.5):
    return _load().or_spalding_yplus(float(up), float(kappa), float(B))


def spalding_newton(R, kappa=0.41, B=5.5, max_iter=1000, tol=1e-14):
    """Returns (u+, iterations, iterates[0..n])."""
    up = np.zeros(1)
    it = np.zeros(max_iter + 1)
    n = _load().or_spalding_newton(float(R), float(kappa), float(B), int(max_iter), float(tol),
                                   _dp(up), _dp(it))
    return up[0], n, it[: n + 1].copy()


def wfb_stress(rho, u, kappa=0.41, B=5.5, y1=1.0, nu=1e-4):
    tw = np.zeros(2)
    _load().or_wfb_stress(float(rho), _dp(_vec(u, 3)), float(kappa), float(B), float(y1),
                          float(nu), _dp(tw))
    return tw


LAW_SPALDING, LAW_LOG, LAW_POWER = 0, 1, 2


def wfb_stress_law(law, rho, u, kappa=0.41, B=5.5, y1=1.0, nu=1e-4):
    tw = np.zeros(2)
    _load().or_wfb_stress_law(int(law), float(rho), _dp(_vec(u, 3)), float(kappa), float(B),
                              float(y1), float(nu), _dp(tw))
    return tw


def loglaw_crossing(kappa=0.41, B=5.5):
    return _load().or_loglaw_crossing(float(kappa), float(B))


def loglaw_uplus(R, kappa=0.41, B=5.5):
    return _load().or_loglaw_uplus(float(R), float(kappa), float(B))


def powerlaw_uplus(R):
    return _load().or_powerlaw_uplus(float(R))


def wall_uplus(law, R, kappa=0.41, B=5.5):
    return _load().or_wall_uplus(int(law), float(R), float(kappa), float(B))


def splitmix64(s: int) -> int:
    return int(_load().or_splitmix64(C.c_uint64(s & 0xFFFFFFFFFFFFFFFF)))


def uniform(seed: int, counter: int) -> float:
    return float(_load().or_uniform(C.c_uint64(seed), C.c_uint64(counter)))


# --------------------------------------------------------- lattice level --

class Lattice:
    """Two-array FP64 lattice; populations are [19][nz][ny][nx]."""

    def __init__(self, nx, ny, nz, tau, cs, force, wall, kappa=0.41, B=5.5, y1=1.0, nu=-1.0,
                 stats_every=0):
        lib = _load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self._lib = lib
        h = lib.or_create(self.nx, self.ny, self.nz, float(tau), float(cs),
                          _dp(_vec(force, 3)), int(wall), float(kappa), float(B), float(y1),
                          float(nu), int(stats_every))
        if not h:
            raise ValueError("oracle: invalid lattice parameters")
        self._h = C.c_void_p(h)

    @classmethod
    def from_case(cls, case, stats_every=0, wall=None):
        L = cls(case.nx, case.ny, case.nz, case.tau, case.cs, case.force,
                case.wall if wall is None else wall, case.kappa, case.b_const, case.y1,
                case.nu_wall, stats_every)
        L.set_wall_law(getattr(case, "wall_law", 0))
        return L

    def close(self):
        if self._h:
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_channel(self, u_mean_x, amp, seed):
        self._lib.or_init_channel(self._h, _dp(_vec(u_mean_x, self.ny)), float(amp),
                                  C.c_uint64(seed))

    def set_populations(self, f):
        self._lib.or_set_populations(self._h, _dp(_vec(f, 19 * self.n)))

    def populations(self):
        out = np.zeros((19, self.nz, self.ny, self.nx))
        self._lib.or_get_populations(self._h, _dp(out))
        return out

    def moments(self):
        rho = np.zeros((self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        self._lib.or_moments(self._h, _dp(rho), _dp(u))
        return rho, u

    def conservation(self):
        out = np.zeros(4)
        self._lib.or_conservation(self._h, _dp(out))
        return out

    def wall_stress(self):
        out = np.zeros((2, self.nz, self.nx, 2))
        self._lib.or_wall_stress(self._h, _dp(out))
        return out

    def wall_delta_f(self):
        out = np.zeros(2)
        self._lib.or_wall_delta_f(self._h, _dp(out))
        return out

    def plane_stats(self, reset=False):
        out = np.zeros((self.ny, K_STATS))
        w = np.zeros((2, 4))
        ns = C.c_longlong(0)
        self._lib.or_plane_stats(self._h, _dp(out), _dp(w), C.byref(ns), int(bool(reset)))
        return out, w, ns.value

    @property
    def step_count(self):
        return int(self._lib.or_get_step(self._h))

    def step(self, n=1):
        self._lib.or_step(self._h, int(n))

    def set_threads(self, threads):
        """All-cores timing mode (threads > 1): unsampled steps run their planes
        in parallel. Returns the thread count in use (1 without OpenMP)."""
        return int(self._lib.or_set_threads(self._h, int(threads)))

    def set_wall_law(self, law):
        """Wall function of the WFB layer: 0 Spalding, 1 log law, 2 power law."""
        if self._lib.or_set_wall_law(self._h, int(law)) != 0:
            raise ValueError(f"oracle: unknown wall law {law}")

    def set_les(self, collision=0, u_tau=0.0, a_plus=0.0):
        """collision 0 BGK / 1 MRT; van Driest damping when a_plus > 0."""
        self._lib.or_set_les(self._h, int(collision), float(u_tau), float(a_plus))
