"""The allocation-free plane profile (lbm_plane_profile_noalloc).

Callers that cannot allocate device memory at measurement time (a fixed memory
budget, a pool that must not grow, host loops that must not synchronise on an
allocation) get the instantaneous plane sums from a fixed scratch array inside
the library. This file is collected last so that a failure here comes after
every other test has run; it must also pass when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()


def _profile_noalloc(ch):
    import torch
    out = torch.empty((ch.ny, lbm.K_STATS), dtype=torch.float64, device="cuda")
    lbm.lbm_plane_profile_noalloc(ch.handle, out.data_ptr())
    ch.sync()
    return out.cpu().numpy()


def _profile_existing(ch):
    """The same sums through lbm_plane_stats: one sampled step accumulates the
    state it starts from."""
    ch.plane_stats(reset=True)
    ch.set_stats_every(1)
    ch.step(1)
    ch.set_stats_every(0)
    st, _, n = ch.plane_stats(reset=True)
    assert n == 1
    return st


@pytest.mark.parametrize("start", [5, 6])
@pytest.mark.parametrize("layout", [lbm.PULL2, lbm.AA])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_noalloc_profile_matches_plane_stats_twice(precision, layout, start):
    """Two calls in a row on the shared scratch. With the single-lattice AA
    layout the state is stored under a different map after an odd and an even
    number of steps; each comparison advances the state by one step, so either
    start covers both maps."""
    case = workload.CASES["c1"].with_(nx=128, ny=24, nz=10)
    ch = lbm.Channel.from_case(case, precision=precision, layout=layout)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.step(start)
    for _ in range(2):                    # two calls in a row on the shared scratch
        got = _profile_noalloc(ch)
        ref = _profile_existing(ch)       # also advances the state by one step
        for k in range(lbm.K_STATS):
            scale = np.max(np.abs(ref[:, k]))
            assert np.max(np.abs(got[:, k] - ref[:, k])) <= 1e-6 * scale, k
    ch.close()


def test_noalloc_profile_rejects_too_many_planes():
    case = workload.CASES["c1"].with_(nx=2, ny=2049, nz=1)
    ch = lbm.Channel.from_case(case)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_plane_profile_noalloc(ch.handle, 1)
    assert ei.value.code == lbm.LBM_ERR_ARG
    assert "2048" in str(ei.value)
    ch.close()
