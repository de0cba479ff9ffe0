"""Failure detection on the GPU, without a GPU fault.

* A NaN written into the populations from the host (lbm_set_populations) is
  reported by the FP64 conservation reduction as LBM_ERR_DIVERGED, before and
  after it has spread through a few steps.
* The shared-memory pipeline waits of the row-pipelined kernel are bounded by
  a limit the caller can set. With a limit of one clock cycle every wait gives
  up before its row arrives (a bulk copy from DRAM takes far longer): the
  kernel sets its error flag, waits (with the default limit) for the copies it
  has already issued, and returns; lbm_sync reports the timeout once, the
  context stays usable, and with the default limit restored the same handle
  reproduces a clean run bit for bit. Every copy issued in this test is a valid
  one and lands; only the wait is cut short.
"""
import numpy as np
import pytest

from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu

SMALL = workload.CASES["c1"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()


def _channel(case, precision=lbm.FP32, kernel=lbm.KERNEL_AUTO, layout=lbm.PULL2):
    ch = lbm.Channel.from_case(case, precision=precision, layout=layout)
    if kernel != lbm.KERNEL_AUTO:
        ch.set_kernel(kernel)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    return ch


@pytest.mark.parametrize("layout", [lbm.PULL2, lbm.AA])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_nan_population_reported_as_diverged(precision, layout):
    case = SMALL.with_(nx=16, ny=6, nz=4)
    ch = _channel(case, precision, layout=layout)
    ok = ch.conservation()
    assert np.all(np.isfinite(ok))
    f = ch.populations()
    f[7, 2, 0, 5] = np.nan          # one wall-layer population
    ch.set_populations(f)
    with pytest.raises(lbm.LbmError) as ei:
        ch.conservation()
    assert ei.value.code == lbm.LBM_ERR_DIVERGED
    ch.step(3)                      # the NaN spreads; still reported
    with pytest.raises(lbm.LbmError) as ei:
        ch.conservation()
    assert ei.value.code == lbm.LBM_ERR_DIVERGED
    ch.close()


def test_pipeline_wait_timeout_is_reported_once_and_recoverable():
    case = SMALL.with_(nx=128, ny=8, nz=6)
    ch = _channel(case, kernel=lbm.KERNEL_TMA)
    assert ch.kernel == lbm.KERNEL_TMA
    ch.sync()
    ch.set_wait_limit(1)
    ch.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        ch.sync()
    assert ei.value.code == lbm.LBM_ERR_CUDA and "timed out" in str(ei.value)
    ch.sync()                       # reported once, then cleared
    # the context still answers: restore the default limit, restart from the
    # seeded field and compare with a fresh handle
    ch.set_wait_limit(0)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.step(20)
    ch.sync()
    ref = _channel(case, kernel=lbm.KERNEL_TMA)
    ref.step(20)
    ref.sync()
    assert np.array_equal(ch.populations(), ref.populations())
    assert np.array_equal(ch.wall_stress(), ref.wall_stress())
    ch.close()
    ref.close()


def test_wait_limit_on_kernels_without_waits_changes_nothing():
    """The limit only concerns the pipelined kernel: the two-cell kernel has no
    waits and runs unchanged under the smallest limit."""
    case = SMALL.with_(nx=64, ny=8, nz=6)
    a = _channel(case, kernel=lbm.KERNEL_PAIR)
    b = _channel(case, kernel=lbm.KERNEL_PAIR)
    a.set_wait_limit(1)
    a.step(17)
    b.step(17)
    a.sync()
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()
