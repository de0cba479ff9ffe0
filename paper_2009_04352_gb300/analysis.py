"""Validation statistics of the channel runs (Sec. 3.2), computed on the host
from what the library returns: the FP64 plane statistics (lbm_plane_stats) and
the wall-stress plane (lbm_wall_stress). These are post-processing of sampled
data, not part of the per-step update.

  mean_profiles      time- and plane-averaged velocity and Reynolds stresses
  wall_units         y+ and u+ of each layer, both halves folded
  spalding_uplus     u+ of Spalding's law (Eq. 16) for given y+
  eps_uplus          L2 error norm of u+ against Spalding's law (Eq. 19),
                     split into buffer (y+ < 100) and log (y+ >= 100) layers
  loglaw_intercept   b of the log law u+ = ln(y+)/kappa + b (Eq. 20)
  y1plus_pdf         PDF of the first-layer y1+ normalised by its mean and
                     standard deviation (Fig. 7)
"""
from __future__ import annotations

import numpy as np

KAPPA = 0.41
B_SPALDING = 5.5


def mean_profiles(stats: np.ndarray, n_samples: int, nx: int, nz: int) -> dict:
    """Per-layer averages from accumulated plane sums [ny][11] (columns rho,
    u_x, u_y, u_z, u_x^2, u_y^2, u_z^2, u_x u_y, rho u_x, rho u_y, rho u_z).
    Reynolds stresses are <u_i u_j> - <u_i><u_j> over time and plane."""
    m = stats / (float(n_samples) * nx * nz)
    ux, uy, uz = m[:, 1], m[:, 2], m[:, 3]
    return {"rho": m[:, 0], "ux": ux, "uy": uy, "uz": uz,
            "uu": m[:, 4] - ux * ux, "vv": m[:, 5] - uy * uy, "ww": m[:, 6] - uz * uz,
            "uv": m[:, 7] - ux * uy}


def wall_units(ux: np.ndarray, u_tau: float, nu: float, y1: float = 1.0):
    """Fold the two halves of the channel and express the mean streamwise
    velocity in wall units. Layer j (counted from the nearer wall) lies at
    y = y1 + j, the same wall-distance convention as the wall model (the first
    layer at y1). Returns (y+, u+) for the ny // 2 layers of one half."""
    ny = len(ux)
    half = ny // 2
    folded = 0.5 * (ux[:half] + ux[::-1][:half])
    y = y1 + np.arange(half, dtype=np.float64)
    return y * u_tau / nu, folded / u_tau


def spalding_yplus(uplus, kappa: float = KAPPA, B: float = B_SPALDING):
    """Eq. 16: y+ as an explicit function of u+."""
    k = kappa * np.asarray(uplus, dtype=np.float64)
    return k / kappa + np.exp(-kappa * B) * (np.expm1(k) - k - k * k / 2.0 - k ** 3 / 6.0)


def spalding_uplus(yplus, kappa: float = KAPPA, B: float = B_SPALDING):
    """u+ of Spalding's law for given y+ > 0 (bisection of the monotone Eq. 16)."""
    yp = np.atleast_1d(np.asarray(yplus, dtype=np.float64))
    # the root lies below y+ (Eq. 16 gives y+ >= u+) and below the log law
    lo = np.zeros_like(yp)
    hi = np.minimum(yp + 1.0, np.log(np.maximum(yp, 1.0)) / kappa + B + 10.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        below = spalding_yplus(mid, kappa, B) < yp
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def eps_uplus(yplus, uplus, split: float = 100.0) -> dict:
    """Eq. 19 against Spalding's law: sqrt(sum (u+ - u+_S)^2 / sum u+_S^2) over
    the buffer layer (y+ < split), the log layer (y+ >= split) and all points.
    A part with no points is NaN."""
    yp = np.asarray(yplus, dtype=np.float64)
    up = np.asarray(uplus, dtype=np.float64)
    ref = spalding_uplus(yp)

    def norm(mask):
        if not np.any(mask):
            return float("nan")
        return float(np.sqrt(np.sum((up[mask] - ref[mask]) ** 2) / np.sum(ref[mask] ** 2)))

    return {"buffer": norm(yp < split), "log": norm(yp >= split), "all": norm(np.ones_like(yp, dtype=bool))}


def loglaw_intercept(yplus, uplus, kappa: float = KAPPA, ymin: float = 100.0) -> float:
    """Least-squares b of u+ = ln(y+)/kappa + b (Eq. 20) with kappa fixed, over
    the points with y+ >= ymin (the logarithmic layer)."""
    yp = np.asarray(yplus, dtype=np.float64)
    up = np.asarray(uplus, dtype=np.float64)
    sel = yp >= ymin
    if not np.any(sel):
        return float("nan")
    return float(np.mean(up[sel] - np.log(yp[sel]) / kappa))


def y1plus_samples(tau_w: np.ndarray, nu: float, y1: float = 1.0, rho: float = 1.0) -> np.ndarray:
    """Instantaneous first-layer y1+ = y1 u_tau / nu with the local
    u_tau = sqrt(|tau_w| / rho), from a wall-stress plane [2][nz][nx][2]."""
    tw = np.asarray(tau_w, dtype=np.float64)
    mag = np.hypot(tw[..., 0], tw[..., 1]).ravel()
    return y1 * np.sqrt(mag / rho) / nu


def y1plus_pdf(samples, bins: int = 41, span: float = 5.0):
    """PDF of (y1+ - mean) / std (Fig. 7) as (bin centres, density)."""
    s = np.asarray(samples, dtype=np.float64)
    sd = s.std()
    z = (s - s.mean()) / (sd if sd > 0 else 1.0)
    hist, edges = np.histogram(z, bins=bins, range=(-span, span), density=True)
    return 0.5 * (edges[1:] + edges[:-1]), hist
