"""Batched ensemble: one persistent launch per step over all members' tiles.

Each member must evolve exactly as the same channel run alone (the batch runs
the two-cell tile code of the single-channel kernel), and therefore as the
oracle within the parity bounds."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu

BASE = workload.CASES["c1"]
MEMBERS = [BASE.with_(nx=64, ny=8, nz=6, wall=workload.WALL_WFB, seed=11),
           BASE.with_(nx=130, ny=6, nz=4, wall=workload.WALL_BB, seed=12, tau=0.55),
           BASE.with_(nx=34, ny=2, nz=3, wall=workload.WALL_FREESLIP, seed=13),
           workload.derive_channel("m3", 96, 24, 48, 395.0, seed=14)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def _init(ch, case):
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_batch_members_equal_single_channels(precision):
    b = lbm.Batch(MEMBERS, precision=precision)
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.set_stats_every(3)
    b.step(40)
    for i, c in enumerate(MEMBERS):
        ch = lbm.Channel.from_case(c, precision=precision)
        ch.set_kernel(lbm.KERNEL_PAIR)          # the tile form the batch runs
        _init(ch, c)
        ch.set_stats_every(3)
        ch.step(40)
        assert np.array_equal(b.members[i].populations(), ch.populations()), i
        assert np.array_equal(b.members[i].wall_stress(), ch.wall_stress()), i
        sb, wb, nb = b.members[i].plane_stats()
        sc, wc, nc = ch.plane_stats()
        assert nb == nc == 14
        # the FP64 reductions may sum in another order (tiles of another width)
        assert np.allclose(sb, sc, rtol=1e-12, atol=1e-12 * np.max(np.abs(sc)))
        assert np.allclose(wb, wc, rtol=1e-12, atol=1e-12 * np.max(np.abs(wc)))
        ch.close()
    b.close()


def test_batch_member_matches_oracle():
    b = lbm.Batch(MEMBERS)
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.step(20)
    for i in (1, 3):
        c = MEMBERS[i]
        L = oracle.Lattice.from_case(c)
        L.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
        L.step(20)
        _, u_o = L.moments()
        _, u_g = b.members[i].moments()
        assert np.max(np.abs(u_g - u_o)) <= 1e-5 * np.max(np.abs(u_o)), i
    b.close()


def test_batch_autotune_and_configs():
    b = lbm.Batch(MEMBERS)
    ms = b.autotune(steps=3)
    assert ms > 0
    cfg = b.config()
    assert cfg["threads"] in (64, 128) and cfg["grid"] >= 1 and cfg["tiles"] > 0
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.set_config(64, 2)
    b.step(9)
    b.set_config(128, 0)
    b.step(8)
    ref = lbm.Channel.from_case(MEMBERS[3])
    _init(ref, MEMBERS[3])
    ref.step(17)
    assert np.array_equal(b.members[3].populations(), ref.populations())
    ref.close()
    b.close()


def test_batch_member_cannot_step_alone():
    b = lbm.Batch(MEMBERS[:2])
    with pytest.raises(lbm.LbmError) as ei:
        b.members[0].step(1)
    assert ei.value.code == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError):
        b.members[0].set_kernel(lbm.KERNEL_CELL)
    assert b.cells == sum(c.cells for c in MEMBERS[:2])
    b.close()
