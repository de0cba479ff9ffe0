"""Time-averaged statistics of long channel runs against the FP64 oracle:
the mean streamwise velocity profile u(y) (u+ = u / u_tau), the mean wall
stress and the streamwise normal stress, time- and plane-averaged as in
Sec. 3.1 (each wall-normal layer averaged over time, then over its plane).

1. The 64 x 32 x 32 parity channel (tau0 = 0.52), 1000 steps: a viscous run
   that decays; every profile within 1%.
2. The Re_tau 640 channel 256 x 64 x 128 (tau0 = 0.500282, WFB walls), 40000
   steps (2.3 eddy turnovers D / u_tau), samples every 10 steps, against the
   oracle's statistics stored in tests/golden/c2_statistics.txt (written by
   tests/golden/make_c2_statistics.py, which runs only the oracle). Over the
   first 20000 steps the runs stay close to one another; after that the flow
   has become chaotic, two runs whose initial fields differ by one part in a
   million decorrelate, and only statistics can agree. In both windows the
   time-averaged u+ profile and the mean wall stress of both walls match the
   oracle within 1% (FP32 and FP16 storage); so does the streamwise normal
   stress <u'u'> in FP32 storage.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import _log

pytestmark = pytest.mark.gpu

STEPS = 1000
EVERY = 10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_statistics.txt")


@pytest.fixture(scope="module")
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def oracle_stats(_cuda):
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


def _read_golden():
    cells = None
    samples, planes, walls = {}, {}, {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        if tok[0] == "cells_per_plane":
            cells = int(tok[1])
        elif tok[0] == "samples":
            samples[int(tok[1])] = int(tok[2])
        elif tok[0] == "plane":
            planes[(int(tok[1]), int(tok[2]))] = [float(v) for v in tok[3:]]
        elif tok[0] == "wall":
            walls[(int(tok[1]), int(tok[2]))] = [float(v) for v in tok[3:]]
    nwin = len(samples)
    ny = max(y for _, y in planes) + 1
    P = np.array([[planes[(w, y)] for y in range(ny)] for w in range(nwin)])     # [win][y][rho, ux, ux2]
    Wl = np.array([[walls[(w, k)] for k in range(2)] for w in range(nwin)])      # [win][wall][tx, |t|]
    return cells, np.array([samples[w] for w in range(nwin)]), P, Wl


def _window(P, Wl, n, cells, lo, hi):
    """Time- and plane-averaged u_x(y), <u'u'>(y), mean tau_w,x and |tau_w| per
    wall over the windows [lo, hi)."""
    ns = n[lo:hi].sum() * cells
    s = P[lo:hi].sum(axis=0)
    ux = s[:, 1] / ns
    uu = s[:, 2] / ns - ux ** 2
    w = Wl[lo:hi].sum(axis=0) / ns
    return ux, uu, w


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_long_chaotic_run_statistics_match_oracle(_cuda, precision):
    case = workload.CASES["c2"]
    cells, n_o, P_o, W_o = _read_golden()
    assert cells == case.nx * case.nz
    nwin = len(n_o)
    window = 10000
    ch = lbm.Channel.from_case(case, precision=precision)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.set_stats_every(EVERY)
    P_g, W_g, n_g = [], [], []
    for _ in range(nwin):
        ch.step(window)
        st, w, ns = ch.plane_stats(reset=True)
        P_g.append(st[:, [0, 1, 4]])
        W_g.append(w[:, [0, 2]])
        n_g.append(ns)
    ch.close()
    P_g, W_g, n_g = np.array(P_g), np.array(W_g), np.array(n_g)
    assert np.array_equal(n_g, n_o)
    u_tau = case.u_tau
    for lo, hi in ((0, nwin // 2), (nwin // 2, nwin)):
        ux_o, uu_o, w_o = _window(P_o, W_o, n_o, cells, lo, hi)
        ux_g, uu_g, w_g = _window(P_g, W_g, n_g, cells, lo, hi)
        up_o, up_g = ux_o / u_tau, ux_g / u_tau
        err = {"u+": float(np.max(np.abs(up_g - up_o)) / np.max(np.abs(up_o))),
               "tau_w": float(np.max(np.abs(w_g - w_o) / np.abs(w_o))),
               "uu": float(np.max(np.abs(uu_g - uu_o)) / np.max(uu_o))}
        _log(("c2 long run", lo, hi), precision, err, {})
        assert err["u+"] <= 0.01, (lo, hi, err)
        assert err["tau_w"] <= 0.01, (lo, hi, err, w_g, w_o)
        if precision == lbm.FP32:
            assert err["uu"] <= 0.01, (lo, hi, err)
