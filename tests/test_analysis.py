"""Validation statistics (Eqs. 16, 19, 20; Fig. 7) pinned against the oracle's
Spalding law and constructed cases with known answers."""
import math

import numpy as np
import pytest

from paper_2009_04352_gb300 import analysis


def test_spalding_inverse_matches_oracle(oracle_lib):
    ups = np.array([0.05, 0.5, 3.0, 8.0, 12.0, 17.0, 22.0, 27.0])
    yps = np.array([oracle_lib.spalding_yplus(u) for u in ups])
    assert np.allclose(analysis.spalding_yplus(ups), yps, rtol=1e-12, atol=1e-14)
    assert np.allclose(analysis.spalding_uplus(yps), ups, rtol=1e-10, atol=1e-12)


def test_eps_uplus_zero_on_the_law_and_scaled_error(oracle_lib):
    ups = np.linspace(2.0, 28.0, 40)
    yps = np.array([oracle_lib.spalding_yplus(u) for u in ups])
    e = analysis.eps_uplus(yps, ups)
    assert e["all"] < 1e-10 and e["buffer"] < 1e-10 and e["log"] < 1e-10
    e = analysis.eps_uplus(yps, 1.05 * ups)      # 5% everywhere -> 0.05 in every part
    for k in ("buffer", "log", "all"):
        assert e[k] == pytest.approx(0.05, rel=1e-8)
    assert (yps < 100).any() and (yps >= 100).any()


def test_loglaw_intercept_recovers_b():
    yp = np.logspace(2, 4, 30)
    for b in (5.4, -4.1, 6.6):
        up = np.log(yp) / 0.41 + b
        assert analysis.loglaw_intercept(yp, up) == pytest.approx(b, abs=1e-12)
    assert math.isnan(analysis.loglaw_intercept(np.array([10.0]), np.array([10.0])))


def test_wall_units_fold_and_scale():
    ux = np.array([1.0, 2.0, 3.0, 3.0, 2.2, 0.8])
    yp, up = analysis.wall_units(ux, u_tau=0.5, nu=0.1, y1=1.0)
    assert np.allclose(yp, [5.0, 10.0, 15.0])
    assert np.allclose(up, [1.8, 4.2, 6.0])


def test_y1plus_pdf_of_gaussian_samples():
    rng = np.random.default_rng(0)
    s = 30.0 + 4.0 * rng.standard_normal(200000)
    x, p = analysis.y1plus_pdf(s, bins=41, span=5.0)
    ref = np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)
    assert np.max(np.abs(p - ref)) < 0.02
    assert np.sum(p) * (x[1] - x[0]) == pytest.approx(1.0, abs=1e-3)


def test_y1plus_samples_from_wall_stress():
    tw = np.zeros((2, 3, 4, 2))
    tw[..., 0] = -4e-6
    tw[..., 1] = 3e-6                             # |tau_w| = 5e-6
    s = analysis.y1plus_samples(tw, nu=1e-4, y1=1.0)
    assert s.shape == (24,) and np.allclose(s, math.sqrt(5e-6) / 1e-4)


def test_mean_profiles_from_oracle_stats(oracle_lib):
    L = oracle_lib.Lattice(8, 6, 4, 0.55, 0.1, (1e-6, 0, 0), 1, stats_every=1)
    j = np.arange(6)
    L.init_channel(0.02 * np.minimum(j + 0.5, 6 - j - 0.5) / 3, 1e-3, 3)
    snaps = []
    for _ in range(4):
        snaps.append(L.moments())
        L.step(1)
    st, _, n = L.plane_stats()
    prof = analysis.mean_profiles(st, n, 8, 4)
    u = np.stack([s[1] for s in snaps])            # [t][3][nz][ny][nx]
    ux_mean = u[:, 0].mean(axis=(0, 1, 3))
    uu = (u[:, 0] ** 2).mean(axis=(0, 1, 3)) - ux_mean ** 2
    assert np.allclose(prof["ux"], ux_mean, rtol=1e-12, atol=1e-16)
    assert np.allclose(prof["uu"], uu, rtol=1e-9, atol=1e-16)
