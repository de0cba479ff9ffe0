"""Shared parity bounds of the GPU tests (imported by the test modules; not a
test module itself).

The bound for every compared quantity is the task's relative L_inf tolerance,
1e-5 for FP32 storage and 5e-3 for FP16 storage, or K_FLOOR = 3 times the
measured storage-rounding floor of that quantity, whichever is larger. The
factor covers the GPU's own FP32 arithmetic (a few roundings per update on top
of the one storage rounding); measured GPU/floor ratios stay below 2.7 for the
density deviation at tau0 -> 1/2, the worst case, and below 2 elsewhere. The floor is the
error that storage rounding alone causes: the FP64 oracle is run with its
population deviations f_a - w_a rounded to the storage precision after the
initial field and after every step, the one rounding the GPU applies when it
stores a step, and compared with the plain oracle. For the density deviation
rho - 1 the floor also rounds rho to FP32, the precision in which the library
returns it (near 1 that output rounding, not the storage, dominates in FP32).

Bounce-back wall stress is the difference of two stored populations
(-2 (f*_b - f*_b') per component, the momentum the reflection returns), 15 to
60 times smaller than the largest population deviation in these channels, so
its bound is the one the population bound implies:
  |tau_gpu - tau_oracle| <= 4 * bound(f - w) * max |f - w|_oracle.
"""
from __future__ import annotations

import functools
import os

import numpy as np

import oracle
from paper_2009_04352_gb300 import lbm, workload

TOL = {lbm.FP32: 1e-5, lbm.FP16_SHIFTED: 5e-3}
STORAGE = {lbm.FP32: np.float32, lbm.FP16_SHIFTED: np.float16}
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None, None, None]


def rel(got, ref):
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(np.asarray(got, dtype=np.float64) - ref)) / max(scale, 1e-300))


K_FLOOR = 3.0


def bound(precision, floor):
    return max(TOL[precision], K_FLOOR * floor)


def _log(tag, precision, err, floor_c):
    path = os.environ.get("LBM_PARITY_LOG")
    if path:
        import json
        with open(path, "a") as fh:
            fh.write(json.dumps({"tag": str(tag), "precision": precision, "err": err, "floor": floor_c}) + "\n")


def _round_state(L, dtype):
    f = L.populations()
    f -= W
    f[...] = f.astype(dtype)
    f += W
    L.set_populations(f)


def reference(case, checkpoints, wall=None, les=None, rounding=None, stats_every=0):
    """Oracle state at each checkpoint: rho, u, tau_w, populations, the
    conservation sums and plane statistics. les = (collision, u_tau, a_plus).
    rounding = lbm.FP32 / lbm.FP16_SHIFTED rounds the deviations to that
    storage after the initial field and after every step. Cached per
    argument set."""
    return _reference(case, tuple(checkpoints), case.wall if wall is None else wall,
                      None if les is None else tuple(les), rounding, stats_every)


@functools.lru_cache(maxsize=None)
def _reference(case, checkpoints, wall, les, rounding, stats_every):
    L = oracle.Lattice.from_case(case, stats_every=stats_every, wall=wall)
    L.set_threads(os.cpu_count() or 1)   # bitwise the serial oracle (pinned on CPU)
    if les is not None:
        L.set_les(*les)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    if rounding is not None:
        _round_state(L, STORAGE[rounding])
    out = {}
    t = 0
    for c in checkpoints:
        if rounding is None:
            L.step(c - t)
        else:
            for _ in range(c - t):
                L.step(1)
                _round_state(L, STORAGE[rounding])
        t = c
        rho, u = L.moments()
        out[c] = dict(rho=rho, u=u, tw=L.wall_stress(), f=L.populations(), cons=L.conservation(),
                      stats=L.plane_stats())
    L.close()
    return out


def floors(case, checkpoints, precision, wall=None, les=None):
    """Storage-rounding floor of u, rho - 1 (rho returned in FP32), f - w and
    tau_w at each checkpoint. Cached per argument set."""
    return _floors(case, tuple(checkpoints), precision, case.wall if wall is None else wall,
                   None if les is None else tuple(les))


@functools.lru_cache(maxsize=None)
def _floors(case, checkpoints, precision, wall, les):
    ref = reference(case, checkpoints, wall, les)
    em = reference(case, checkpoints, wall, les, rounding=precision)
    out = {}
    for c in checkpoints:
        r, e = ref[c], em[c]
        rho32 = e["rho"].astype(np.float32).astype(np.float64)
        out[c] = dict(u=rel(e["u"], r["u"]), rho=rel(rho32 - 1.0, r["rho"] - 1.0),
                      f=rel(e["f"] - W, r["f"] - W),
                      tw=rel(e["tw"], r["tw"]) if np.any(r["tw"]) else 0.0)
    return out


def check_state(ch, ref_c, floor_c, precision, wall, populations=False, tag=""):
    """Compare the channel's current state with the oracle's (ref_c) under the
    bounds above; returns the measured errors."""
    rho, u = ch.moments()
    tw = ch.wall_stress()
    err = {"u": rel(u, ref_c["u"]), "rho": rel(rho - 1.0, ref_c["rho"] - 1.0)}
    fb = ref_c["f"] - W
    if wall not in (workload.WALL_FREESLIP, workload.WALL_BB):
        err["tw"] = rel(tw, ref_c["tw"])
    if populations:
        err["f"] = rel(ch.populations() - W, fb)
    _log(tag, precision, err, floor_c)
    assert err["u"] <= bound(precision, floor_c["u"]), (tag, err)
    assert err["rho"] <= bound(precision, floor_c["rho"]), (tag, err, floor_c["rho"])
    if wall == workload.WALL_FREESLIP:
        assert np.all(tw == 0.0), tag
    elif wall == workload.WALL_BB:
        dtw = float(np.max(np.abs(tw.astype(np.float64) - ref_c["tw"])))
        err["tw_abs"] = dtw
        assert dtw <= 4.0 * bound(precision, floor_c["f"]) * np.max(np.abs(fb)), (tag, err)
    else:
        assert err["tw"] <= bound(precision, floor_c["tw"]), (tag, err, floor_c["tw"])
    if populations:
        assert err["f"] <= bound(precision, floor_c["f"]), (tag, err, floor_c["f"])
    return err
