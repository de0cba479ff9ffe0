"""The single-channel kernel-form autotuner (lbm_autotune, autotune.tune_channel):
it times every form the grid allows, keeps the fastest, and the channel it
leaves behind still computes the oracle's update."""
import os

import pytest

import oracle
from paper_2009_04352_gb300 import autotune, lbm, workload
from parity import check_state, floors, reference

pytestmark = pytest.mark.gpu

CASE = workload.CASES["c1"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def _allowed(case, precision):
    ks = {lbm.KERNEL_CELL}
    if case.nx % 2 == 0:
        ks.add(lbm.KERNEL_PAIR)
    if case.nx % 64 == 0:
        ks.add(lbm.KERNEL_TMA)
    if case.nx % 4 == 0 and precision == lbm.FP16_SHIFTED:
        ks.add(lbm.KERNEL_QUAD)
    return ks


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_autotune_picks_an_allowed_form_and_stays_on_the_oracle(precision):
    ch = lbm.Channel.from_case(CASE, precision=precision)
    kernel, ms = ch.autotune(8)
    assert kernel in _allowed(CASE, precision) and ch.kernel == kernel
    assert ms > 0.0
    assert ch.step_count == len(_allowed(CASE, precision)) * (8 + 2)
    ch.init_channel(workload.u_mean_profile(CASE), workload.noise_amplitude(CASE), CASE.seed)
    ch.step(100)
    check_state(ch, reference(CASE, (100,))[100], floors(CASE, (100,), precision)[100], precision, CASE.wall,
                populations=True, tag=("autotune", kernel))
    ch.close()


def test_autotune_odd_grid_has_one_form():
    case = CASE.with_(nx=37, ny=6, nz=5)
    ch = lbm.Channel.from_case(case)
    kernel, _ = ch.autotune(2)
    assert kernel == lbm.KERNEL_CELL
    ch.close()


def test_tune_channel_caches_the_choice(tmp_path):
    path = os.path.join(tmp_path, "tune.json")
    a = lbm.Channel.from_case(CASE, precision=lbm.FP16_SHIFTED)
    first = autotune.tune_channel(a, cache_path=path, steps=4)
    assert not first["cached"]
    b = lbm.Channel.from_case(CASE, precision=lbm.FP16_SHIFTED)
    b.set_kernel(lbm.KERNEL_CELL)
    second = autotune.tune_channel(b, cache_path=path)
    assert second["cached"] and b.kernel == first["kernel"]
    a.close()
    b.close()
