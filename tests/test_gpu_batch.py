"""Batched ensemble: the persistent form (one launch per step over all
members' two-cell tiles) and the member-grid form (every member's own
single-channel kernels, captured for all members as one graph per chunk).

Each member must evolve exactly as the same channel run alone (the two-cell
kernel's arithmetic in both forms: the FP16 four-cell kernel computes the
same bits), and therefore as the oracle within the parity bounds
(tests/parity.py)."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import check_state, floors, reference

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
        # the members run the kernel their grid selects (four cells per thread
        # for FP16 where nx allows): the same cell values, added per thread and
        # per warp in FP32 in another order than the two-cell tiles, so the
        # sums agree to a few FP32 roundings of the warp sums
        for got, ref in ((sb, sc), (wb, wc)):
            scale = np.max(np.abs(ref), axis=0)
            assert np.all(np.abs(got - ref) <= 1e-6 * scale), np.max(np.abs(got - ref) / scale)
        ch.close()
    b.close()


@pytest.mark.parametrize("form", [lbm.BATCH_PERSISTENT, lbm.BATCH_MEMBER_GRIDS])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_batch_members_match_oracle(precision, form):
    """Every member against the FP64 oracle after 20 steps: velocity, density,
    populations and wall stress."""
    b = lbm.Batch(MEMBERS, precision=precision)
    b.set_form(form)
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.step(20)
    for i, c in enumerate(MEMBERS):
        check_state(b.members[i], reference(c, (20,))[20], floors(c, (20,), precision)[20], precision, c.wall,
                    populations=True, tag=("batch", form, i))
    b.close()


@pytest.mark.parametrize("streams", [1, 3])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_batch_member_grids_equal_single_channels(precision, streams):
    """Member-grid form: each member is the channel run alone with the kernel
    its grid selects (four-cell for FP16 where nx allows, else two-cell),
    statistics included."""
    b = lbm.Batch(MEMBERS, precision=precision)
    b.set_form(lbm.BATCH_MEMBER_GRIDS, streams)
    assert b.form == lbm.BATCH_MEMBER_GRIDS and b.config()["streams"] == streams
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.set_stats_every(3)
    b.step(40)
    for i, c in enumerate(MEMBERS):
        ch = lbm.Channel.from_case(c, precision=precision)
        _init(ch, c)
        ch.set_stats_every(3)
        ch.step(40)
        assert np.array_equal(b.members[i].populations(), ch.populations()), i
        assert np.array_equal(b.members[i].wall_stress(), ch.wall_stress()), i
        sb, wb, nb = b.members[i].plane_stats()
        sc, wc, nc = ch.plane_stats()
        assert nb == nc == 14
        assert np.array_equal(sb, sc) and np.array_equal(wb, wc), i
        ch.close()
    b.close()


def test_batch_forms_switch_between_steps():
    """The state does not depend on the form: persistent steps, then member-grid
    steps, equal the same steps of each channel alone (FP16: the four-cell and
    two-cell kernels give the same bits)."""
    for precision in (lbm.FP32, lbm.FP16_SHIFTED):
        b = lbm.Batch(MEMBERS, precision=precision)
        for m, c in zip(b.members, MEMBERS):
            _init(m, c)
        b.step(5)
        b.set_form(lbm.BATCH_MEMBER_GRIDS, 2)
        b.step(6)
        b.set_form(lbm.BATCH_PERSISTENT)
        b.step(3)
        for i, c in enumerate(MEMBERS):
            ref = lbm.Channel.from_case(c, precision=precision)
            ref.set_kernel(lbm.KERNEL_PAIR)
            _init(ref, c)
            ref.step(14)
            assert np.array_equal(b.members[i].populations(), ref.populations()), (precision, i)
            assert np.array_equal(b.members[i].wall_stress(), ref.wall_stress()), (precision, i)
            ref.close()
        b.close()


def test_batch_form_rules():
    b = lbm.Batch(MEMBERS[:2])
    assert b.form == lbm.BATCH_MEMBER_GRIDS
    for form, streams in ((3, 0), (0, 0), (lbm.BATCH_MEMBER_GRIDS, 33), (lbm.BATCH_MEMBER_GRIDS, -1)):
        with pytest.raises(lbm.LbmError):
            b.set_form(form, streams)
    b.set_form(lbm.BATCH_MEMBER_GRIDS)
    assert b.config()["streams"] == 8
    b.close()


def test_batch_autotune_searches_both_forms():
    b = lbm.Batch(MEMBERS, precision=lbm.FP16_SHIFTED)
    ms = b.autotune(steps=3)
    cfg = b.config()
    assert ms > 0 and cfg["form"] in (lbm.BATCH_PERSISTENT, lbm.BATCH_MEMBER_GRIDS)
    for m, c in zip(b.members, MEMBERS):
        _init(m, c)
    b.step(7)
    ref = lbm.Channel.from_case(MEMBERS[3], precision=lbm.FP16_SHIFTED)
    ref.set_kernel(lbm.KERNEL_PAIR)
    _init(ref, MEMBERS[3])
    ref.step(7)
    assert np.array_equal(b.members[3].populations(), ref.populations())
    ref.close()
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
