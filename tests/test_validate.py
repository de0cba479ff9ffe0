"""Host logic of the validation runner (no GPU): the Table 1 grids and the
summary statistics, fed with plane sums of known profiles."""
import math

import numpy as np
import pytest

from paper_2009_04352_gb300 import analysis, validate


@pytest.mark.parametrize("name,ny_half", [("A20", 20), ("A40", 40), ("B40", 40), ("B80", 80)])
def test_table1_grids(name, ny_half):
    """Table 1: 2 pi D x 2D x pi D at D/dx = 20, 40, 80; y+ of the first
    layer = Re_tau dx / D (32, 16, 50, 25)."""
    halfway = validate.table1_case(name, "wfb", 1.0)
    node = validate.table1_case(name, "wfb_node", 1.0)
    assert halfway.ny == 2 * ny_half and node.ny == 2 * ny_half + 1
    assert halfway.half_height == node.half_height == ny_half
    assert abs(halfway.nx - 2 * math.pi * ny_half) <= 1 and abs(halfway.nz - math.pi * ny_half) <= 1
    re_tau = validate.TABLE1[name][0]
    assert halfway.u_tau / halfway.nu == pytest.approx(re_tau / ny_half)   # y+ of one lattice spacing
    assert node.u_tau / node.nu == pytest.approx(re_tau / ny_half)


def _stats_of_profile(case, ux_layers, n=3):
    """Plane sums [ny][11] of n samples of a steady profile (rho = 1)."""
    st = np.zeros((case.ny, 11))
    cells = case.nx * case.nz * n
    st[:, 0] = cells
    st[:, 1] = cells * ux_layers
    st[:, 4] = cells * ux_layers ** 2
    st[:, 8] = cells * ux_layers
    return st


@pytest.mark.parametrize("wall", ["wfb", "wfb_node"])
def test_summary_of_a_spalding_profile(wall):
    """A profile on Spalding's law gives eps_u+ ~ 0 everywhere and the log-layer
    intercept of Spalding's law itself (its outer asymptote has b = B = 5.5,
    approached from below at finite y+); the measured u_tau is recovered from the
    wall sums."""
    case = validate.table1_case("B40", wall, 1.0)
    j = np.arange(case.ny, dtype=np.float64)
    if wall == "wfb_node":
        d = np.minimum(j, case.ny - 1 - j)
    else:
        d = np.minimum(j + 0.5, case.ny - j - 0.5)
    ux = case.u_tau * analysis.spalding_uplus(d * case.u_tau / case.nu)
    stats = _stats_of_profile(case, ux)
    n = 3
    tau = case.u_tau ** 2
    wstats = np.array([[-tau * case.nx * case.nz * n, 0, tau * case.nx * case.nz * n, 0]] * 2)
    taus = np.zeros((4, 2, case.nz, case.nx, 2))
    taus[..., 0] = -tau * (1 + 0.1 * np.random.default_rng(1).standard_normal((4, 2, case.nz, case.nx)))
    out = validate.summarise(case, stats, wstats, n, taus, {})
    assert out["eps_uplus"]["all"] < 1e-9
    assert 5.0 < out["loglaw_b"] < 5.5
    assert out["u_tau_measured"] == pytest.approx(case.u_tau, rel=1e-12)
    assert out["first_layer"]["yplus"] == pytest.approx((1.0 if wall == "wfb_node" else 0.5) * 2003.0 / 40)
    assert abs(out["y1plus"]["skew"]) < 0.5


def test_summary_flags_a_slow_profile():
    """A profile 10% below Spalding's law reads as eps_u+ = 0.1 and a lower b."""
    case = validate.table1_case("A20", "wfb", 1.0)
    j = np.arange(case.ny, dtype=np.float64)
    d = np.minimum(j + 0.5, case.ny - j - 0.5)
    ux = 0.9 * case.u_tau * analysis.spalding_uplus(d * case.u_tau / case.nu)
    out = validate.summarise(case, _stats_of_profile(case, ux), np.zeros((2, 4)), 3,
                             np.full((1, 2, case.nz, case.nx, 2), 1e-7), {})
    assert out["eps_uplus"]["all"] == pytest.approx(0.1, rel=1e-6)
    assert out["loglaw_b"] < 4.5
