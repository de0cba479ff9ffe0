"""Time-averaged statistics of a longer run against the oracle: the mean
streamwise velocity profile and the mean wall stress within 1% (the statistics
of Sec. 3.1: time averaging of each wall-normal layer, then plane averaging)."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu

STEPS = 1000
EVERY = 10


@pytest.fixture(scope="module")
def oracle_stats():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()
    case = workload.CASES["c1"]
    L = oracle.Lattice.from_case(case, stats_every=EVERY)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    L.step(STEPS)
    st, w, n = L.plane_stats()
    L.close()
    return case, st, w, n


def _profiles(st, w, n, case):
    cells = case.nx * case.nz
    ux = st[:, 1] / (n * cells)
    urms = np.sqrt(np.maximum(st[:, 4] / (n * cells) - ux ** 2, 0.0))
    tw = w[:, 0] / (n * cells)           # mean tau_w,x per wall
    return ux, urms, tw


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_time_averaged_profiles_match_oracle(oracle_stats, precision):
    case, st_o, w_o, n_o = oracle_stats
    ch = lbm.Channel.from_case(case, precision=precision)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.set_stats_every(EVERY)
    ch.step(STEPS)
    st_g, w_g, n_g = ch.plane_stats()
    ch.close()
    assert n_g == n_o == STEPS // EVERY
    ux_o, urms_o, tw_o = _profiles(st_o, w_o, n_o, case)
    ux_g, urms_g, tw_g = _profiles(st_g, w_g, n_g, case)
    assert np.max(np.abs(ux_g - ux_o)) <= 0.01 * np.max(np.abs(ux_o))
    assert np.max(np.abs(tw_g - tw_o)) <= 0.01 * np.max(np.abs(tw_o))
    assert np.max(np.abs(urms_g - urms_o)) <= 0.01 * np.max(urms_o)
