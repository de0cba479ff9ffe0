"""Seeded synthetic channel workloads: grids, parameters and initial-field inputs.

This module is the only code shared by the CUDA path and the FP64 oracle. It
holds no part of the lattice update itself: it picks the channel sizes, the
lattice parameters (tau0, body force, wall-model constants) and the smooth mean
profile that seeds the initial field. The per-cell random perturbation is drawn
inside each implementation from the counter-based SplitMix64 generator
(Steele, Lea & Flood 2014), keyed by the seed given here.

Lattice units throughout: dx = dt = 1, c_s^2 = 1/3, rho0 = 1. The channel is
x streamwise (periodic), y wall-normal (walls at y = -1/2 and y = ny - 1/2, so
the half height is D = ny / 2), z spanwise (periodic), as in the paper's
turbulent channel set-up (Sec. 3.1, Fig. 3). With wall nodes (the full-way
form of the WFB) the layers 0 and ny - 1 are the walls and D = (ny - 1) / 2.

Parameter recipe (the paper prints physical settings in Table 1 but no lattice
values): a centreline velocity U_c = 0.04 keeps the lattice Mach number near the
paper's 0.06-0.07; u_tau = U_c / u+(Re_tau) from the log law (Eq. 20 with
b = B = 5.5); nu = u_tau * D / Re_tau; tau0 = 1/2 + 3 nu; F_x = u_tau^2 / D,
the force that balances a wall stress rho * u_tau^2 on both walls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

KAPPA = 0.41          # von Karman constant (Sec. 2.3, after Eq. 16)
B_CONST = 5.5         # Spalding / log-law additive constant (Sec. 2.3)
U_CENTRE = 0.04       # lattice centreline velocity of the synthetic channels
NOISE_FRAC = 0.10     # uniform noise amplitude, fraction of the bulk velocity

WALL_BB = 0
WALL_WFB = 1
WALL_FREESLIP = 2
WALL_WFB_NODE = 3     # full-way WFB on wall nodes at layers 0 and ny - 1
WALL_NAMES = {WALL_BB: "bb", WALL_WFB: "wfb", WALL_FREESLIP: "freeslip", WALL_WFB_NODE: "wfb_node"}


def log_law_uplus(yplus):
    """Two-layer mean profile u+(y+): viscous sublayer u+ = y+ joined to the log
    law u+ = ln(y+)/kappa + B where the two cross (continuous, explicit).

    This is the "log-law mean profile" of the synthetic initial field. It is an
    input recipe, not the wall function the method uses at run time.
    """
    yp = np.asarray(yplus, dtype=np.float64)
    safe = np.maximum(yp, 1.0)
    log_branch = np.log(safe) / KAPPA + B_CONST
    return np.where(yp < 1.0, yp, np.minimum(yp, log_branch))


@dataclass(frozen=True)
class ChannelCase:
    """One synthetic channel: grid, lattice parameters and initial-field recipe."""

    name: str
    nx: int
    ny: int
    nz: int
    re_tau: float                 # shapes the initial profile (y+ = Re_tau d / D)
    tau: float                    # BGK relaxation time tau0 (molecular viscosity)
    cs: float                     # Smagorinsky constant C_s
    force: tuple                  # body force per unit volume (F_x, F_y, F_z)
    wall: int                     # WALL_BB / WALL_WFB / WALL_FREESLIP
    u_tau: float                  # friction velocity used for the profile
    seed: int
    steps: int = 100
    kappa: float = KAPPA
    b_const: float = B_CONST
    y1: float = 1.0               # wall distance used in y+ = y1 u_tau / nu
    nu_wall: float = -1.0         # wall-function viscosity; < 0 means (tau0 - 1/2)/3
    newton_iters: int = 12
    noise_frac: float = NOISE_FRAC
    wall_law: int = 0             # 0 Spalding (Eq. 16), 1 log law, 2 Werner-Wengle power law

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def half_height(self) -> float:
        return (self.ny - 1) / 2.0 if self.wall == WALL_WFB_NODE else self.ny / 2.0

    @property
    def nu(self) -> float:
        return self.nu_wall if self.nu_wall > 0 else (self.tau - 0.5) / 3.0

    def with_(self, **kw) -> "ChannelCase":
        return replace(self, **kw)


def u_mean_profile(case: ChannelCase) -> np.ndarray:
    """Mean streamwise velocity per wall-normal layer j (length ny), FP64."""
    j = np.arange(case.ny, dtype=np.float64)
    if case.wall == WALL_WFB_NODE:   # distance to the nearer wall node (0 on the walls)
        d = np.minimum(j, case.ny - 1 - j)
    else:
        d = np.minimum(j + 0.5, case.ny - j - 0.5)
    yplus = case.re_tau * d / case.half_height
    return case.u_tau * log_law_uplus(yplus)


def noise_amplitude(case: ChannelCase) -> float:
    """Uniform noise half-width: NOISE_FRAC of the bulk (layer-mean) velocity."""
    return float(case.noise_frac * np.mean(u_mean_profile(case)))


def derive_channel(name, nx, ny, nz, re_tau, wall=WALL_WFB, seed=1, steps=100,
                   cs=0.1, u_centre=U_CENTRE) -> ChannelCase:
    """Channel whose tau0 and force follow from Re_tau (recipe in the module doc)."""
    D = (ny - 1) / 2.0 if wall == WALL_WFB_NODE else ny / 2.0
    u_tau = u_centre / float(log_law_uplus(re_tau))
    nu = u_tau * D / re_tau
    tau = 0.5 + 3.0 * nu
    fx = u_tau * u_tau / D
    return ChannelCase(name=name, nx=nx, ny=ny, nz=nz, re_tau=re_tau, tau=tau, cs=cs,
                       force=(fx, 0.0, 0.0), wall=wall, u_tau=u_tau, seed=seed, steps=steps)


def _small_parity_case() -> ChannelCase:
    """64x32x32 at tau0 = 0.52, C_s = 0.1, profile shaped by Re_tau = 640.

    tau0 = 0.52 and Re_tau = 640 cannot both hold at D = 16 (u_tau would be
    0.27, far above the lattice sound speed). The velocity scale is therefore
    taken from U_c = 0.04 (u_tau = U_c / u+(640)) and F_x = u_tau^2 / D, while
    Re_tau = 640 only shapes the initial profile.
    """
    ny = 32
    u_tau = U_CENTRE / float(log_law_uplus(640.0))
    return ChannelCase(name="c1_64x32x32_tau0.52", nx=64, ny=ny, nz=32, re_tau=640.0,
                       tau=0.52, cs=0.1, force=(u_tau * u_tau / (ny / 2.0), 0.0, 0.0),
                       wall=WALL_WFB, u_tau=u_tau, seed=1, steps=500)


CASES = {
    "c1": _small_parity_case(),
    "c2": derive_channel("c2_256x64x128_re640", 256, 64, 128, 640.0, seed=2, steps=20000),
    "c3": derive_channel("c3_512x128x256_re2003", 512, 128, 256, 2003.0, seed=3, steps=50000),
    "c4": derive_channel("c4_1024x256x512_re2003", 1024, 256, 512, 2003.0, seed=4, steps=2000),
}

BATCH_NY = (32, 48, 64, 96, 128)
BATCH_RE = (180.0, 395.0, 640.0, 1000.0, 2003.0)


def batch_cases(n: int = 64, seed: int = 5, wall: int = WALL_WFB, scale: int = 1):
    """Ensemble of independent channels of uneven sizes and Re_tau.

    ny is drawn uniformly from {32, 48, 64, 96, 128} (divided by `scale` for
    small test ensembles), nx = 4 ny, nz = 2 ny, Re_tau uniformly from
    {180, 395, 640, 1000, 2003}; instance i uses seed 5000 + i.
    """
    rng = np.random.default_rng(seed)
    ny_pick = rng.integers(0, len(BATCH_NY), size=n)
    re_pick = rng.integers(0, len(BATCH_RE), size=n)
    out = []
    for i in range(n):
        ny = max(4, BATCH_NY[ny_pick[i]] // scale)
        re = BATCH_RE[re_pick[i]]
        out.append(derive_channel(f"batch{i}_{4*ny}x{ny}x{2*ny}_re{int(re)}", 4 * ny, ny, 2 * ny,
                                  re, wall=wall, seed=5000 + i))
    return out
