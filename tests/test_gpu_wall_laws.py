"""The WFB frame with other wall functions (Sec. 2.3 takes tau_w from any law;
the introduction names the log law and Werner and Wengle's power law besides
Spalding's): the CUDA path against the oracle, per wall cell over a sweep of
R = y1 |u_t| / nu across both branches of each law, over 100 steps of a
channel whose first layer sits in the log region, and through the batch."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import check_state, floors, reference

pytestmark = pytest.mark.gpu

LAWS = [lbm.LAW_SPALDING, lbm.LAW_LOG, lbm.LAW_POWER]
# first layer at y+ ~ 40, R = y+ u+ ~ 500: the log (or power) branch of every law
CHANNEL = workload.derive_channel("wall-law channel 64x32x32", 64, 32, 32, 640.0, seed=21)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b)) / np.max(np.abs(b)))


def _sweep_populations(nx, ny, nz):
    """f = f^eq(rho, u) with the wall-layer |u_t| spanning 1e-5 .. 1e-1 along x
    (R = 10 .. 1e5 at nu = 1e-6), both tangential components, both signs."""
    f = np.empty((19, nz, ny, nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                ut = 10.0 ** (-5.0 + 4.0 * x / (nx - 1))
                ang = 0.7 * z + 0.3 * y
                u = (ut * np.cos(ang), 1e-4 * ((x + z) % 3 - 1), ut * np.sin(ang))
                f[:, z, y, x] = oracle.feq(1.0 + 3e-5 * ((x * 7 + z) % 5), u)
    return f


@pytest.mark.parametrize("kernel", [lbm.KERNEL_PAIR, lbm.KERNEL_CELL, lbm.KERNEL_TMA])
@pytest.mark.parametrize("law", LAWS)
def test_wall_stress_sweep_per_cell(law, kernel):
    """One step from prescribed populations: every wall cell's tau_w equals the
    oracle's law applied to the same cell, to 2e-5 relative (FP32 storage of
    the deviations, the FP32 Newton stop at 1e-7)."""
    nx, ny, nz = 128, 4, 6
    case = workload.CASES["c1"].with_(nx=nx, ny=ny, nz=nz, nu_wall=1e-6, wall_law=law,
                                      force=(0.0, 0.0, 0.0))
    f0 = _sweep_populations(nx, ny, nz)
    L = oracle.Lattice.from_case(case)
    L.set_populations(f0)
    L.step(1)
    tw_ref = L.wall_stress()
    L.close()
    ch = lbm.Channel.from_case(case)
    ch.set_kernel(kernel)
    ch.set_populations(f0)
    ch.step(1)
    tw = ch.wall_stress()
    ch.close()
    mag = np.hypot(tw_ref[..., 0], tw_ref[..., 1])[..., None]
    assert np.all(np.abs(tw - tw_ref) <= 2e-5 * mag + 1e-30)
    # the sweep reaches both branches of the law
    R = 1e-6 ** -1 * 10.0 ** (-5.0 + 4.0 * np.arange(nx) / (nx - 1))
    assert R.min() < 100 and R.max() > 1e4


@pytest.mark.parametrize("kernel", [lbm.KERNEL_PAIR, lbm.KERNEL_CELL, lbm.KERNEL_QUAD, lbm.KERNEL_TMA])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("law", [lbm.LAW_LOG, lbm.LAW_POWER])
def test_wall_law_parity_100_steps(law, precision, kernel):
    if kernel == lbm.KERNEL_QUAD and precision != lbm.FP16_SHIFTED:
        pytest.skip("the four-cell kernel serves FP16 storage only")
    case = CHANNEL.with_(wall_law=law)
    ref = reference(case, (100,))[100]
    fl = floors(case, (100,), precision)[100]
    ch = lbm.Channel.from_case(case, precision=precision)
    ch.set_kernel(kernel)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.step(100)
    check_state(ch, ref, fl, precision, case.wall, populations=True, tag=kernel)
    ch.close()


def test_laws_give_different_stress():
    """The selector is live: the three laws give different wall stress on the
    same log-region channel (and Spalding's matches the default model)."""
    out = {}
    for law in LAWS:
        ch = lbm.Channel.from_case(CHANNEL.with_(wall_law=law))
        ch.init_channel(workload.u_mean_profile(CHANNEL), workload.noise_amplitude(CHANNEL), CHANNEL.seed)
        ch.step(1)
        out[law] = ch.wall_stress()
        ch.close()
    ch = lbm.Channel.from_case(CHANNEL)
    ch.init_channel(workload.u_mean_profile(CHANNEL), workload.noise_amplitude(CHANNEL), CHANNEL.seed)
    ch.step(1)
    assert np.array_equal(ch.wall_stress(), out[lbm.LAW_SPALDING])
    ch.close()
    for a in LAWS:
        for b in LAWS:
            if a < b:
                assert rel(out[a], out[b]) > 1e-3, (a, b)


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_batch_members_with_mixed_laws(precision):
    """Each member of a batch keeps its own wall law: bitwise equal to the same
    channel run alone on the two-cell kernel, and within parity of the oracle."""
    members = [CHANNEL.with_(wall_law=law, seed=31 + law) for law in LAWS]
    b = lbm.Batch(members, precision=precision)
    for m, c in zip(b.members, members):
        m.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
    b.step(30)
    for i, c in enumerate(members):
        ch = lbm.Channel.from_case(c, precision=precision)
        ch.set_kernel(lbm.KERNEL_PAIR)
        ch.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
        ch.step(30)
        assert np.array_equal(b.members[i].populations(), ch.populations()), i
        assert np.array_equal(b.members[i].wall_stress(), ch.wall_stress()), i
        ch.close()
        check_state(b.members[i], reference(c, (30,))[30], floors(c, (30,), precision)[30], precision, c.wall,
                    populations=True, tag=i)
    b.close()
