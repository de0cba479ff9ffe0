"""Validation run of Sec. 3: a turbulent channel advanced on the GPU to a
statistically steady state, then sampled, reporting the statistics of
Sec. 3.2 against Spalding's law: the L2 error norm eps_u+ in the buffer and
logarithmic layers (Eq. 19), the log-law intercept b (Eq. 20), the measured
friction velocity and the first-layer y1+ distribution (Fig. 7).

Grids are the paper's Table 1 cases (domain 2 pi D x 2D x pi D, D/dx = 20,
40 or 80 at Re_tau 640 and 2003); the LES operator is the paper's (MRT,
Smagorinsky C_s = 0.1, van Driest damping with A+ = 26, or none with
--a-plus 0); lattice parameters
follow the synthetic-workload recipe of workload.py (U_c = 0.04). Time is
counted in T = D / u_tau as in Sec. 3.1: statistics are accumulated from
t_spin T to t_end T. Results are normalised with D and the theoretical u_tau,
as the paper does. The wall treatment is one of
  bb        halfway bounce-back,
  wfb       halfway WFB with the wall law at distance y1 (1.0: Table 1's
            first-layer y+, 0.5: the layer centre),
  wfb_node  full-way WFB with wall nodes (first fluid node at distance 1).
Profiles are evaluated at the physical distance of each layer from the wall
(j + 1/2 for halfway walls, j for wall nodes).

    python -m paper_2009_04352_gb300.validate --case A20 --wall wfb --y1 1.0

prints one JSON object. The run uses the CUDA library only; it fails if the
library is not built.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis, workload

# Table 1: (Re_tau, D / dx)
TABLE1 = {"A20": (640.0, 20), "A40": (640.0, 40), "B40": (2003.0, 40), "B80": (2003.0, 80)}
WALLS = {"bb": workload.WALL_BB, "wfb": workload.WALL_WFB, "wfb_node": workload.WALL_WFB_NODE}
A_PLUS = 26.0


def table1_case(name: str, wall: str, y1: float, seed: int = 11, law: int = 0) -> workload.ChannelCase:
    """The Table 1 grid of `name` (nx = 2 pi D, nz = pi D rounded to even
    counts of cells; ny = 2D halfway layers, or 2D + 1 nodes with wall nodes)."""
    re_tau, d = TABLE1[name]
    nx = 2 * int(round(math.pi * d))
    nz = 2 * int(round(math.pi * d / 2))
    kind = WALLS[wall]
    ny = 2 * d + 1 if kind == workload.WALL_WFB_NODE else 2 * d
    c = workload.derive_channel(f"{name}_{wall}_{nx}x{ny}x{nz}", nx, ny, nz, re_tau, wall=kind, seed=seed)
    return c.with_(y1=y1, wall_law=law)


def run(case: workload.ChannelCase, t_spin: float, t_end: float, samples_per_t: float = 10.0,
        snapshots: int = 24, precision: int = 0, stream=None, a_plus: float = A_PLUS) -> dict:
    from . import lbm
    T = case.half_height / case.u_tau
    n_spin = int(round(t_spin * T))
    n_end = int(round(t_end * T))
    every = max(1, int(round(T / samples_per_t)))
    ch = lbm.Channel.from_case(case, precision=precision, stream=stream)
    ch.set_les(lbm.COLLISION_MRT, case.u_tau if a_plus > 0 else 0.0, a_plus)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    t0 = time.perf_counter()
    ch.step(n_spin)
    ch.plane_stats(reset=True)
    ch.set_stats_every(every)
    # sample window in `snapshots` pieces; the wall stress plane of each piece
    # end feeds the y1+ distribution
    n_sample = n_end - n_spin
    taus = []
    done = 0
    for k in range(snapshots):
        seg = (n_sample * (k + 1)) // snapshots - done
        ch.step(seg)
        done += seg
        taus.append(ch.wall_stress().astype(np.float64))
    ch.sync()
    wall_s = time.perf_counter() - t0
    stats, wstats, ns = ch.plane_stats()
    try:
        cons = ch.conservation()
    except lbm.LbmError:          # a run that diverged reports non-finite sums
        cons = np.array([np.nan])
    ch.close()
    return summarise(case, stats, wstats, ns, np.stack(taus), dict(
        steps=n_end, spin_up_steps=n_spin, sample_every=every, samples=int(ns), T_steps=T,
        wall_seconds=wall_s, MLUPS=case.cells * n_end / wall_s / 1e6, finite=bool(np.all(np.isfinite(cons)))))


def summarise(case, stats, wstats, ns, taus, run_info) -> dict:
    prof = analysis.mean_profiles(stats, ns, case.nx, case.nz)
    ux = prof["ux"]
    node = case.wall == workload.WALL_WFB_NODE
    if node:
        ux, y_first = ux[1:-1], 1.0     # fluid layers 1 .. ny - 2, node j at distance j
    else:
        y_first = 0.5                   # layer j at j + 1/2
    yplus, uplus = analysis.wall_units(ux, case.u_tau, case.nu, y_first)
    eps = analysis.eps_uplus(yplus, uplus)
    b = analysis.loglaw_intercept(yplus, uplus)
    # measured friction velocity: mean streamwise wall stress of both walls
    cells = ns * case.nx * case.nz
    tau_x = -0.5 * (wstats[0, 0] + wstats[1, 0]) / cells if cells else float("nan")
    u_tau_meas = math.sqrt(tau_x) if tau_x > 0 else float("nan")
    s = analysis.y1plus_samples(taus, case.nu, y_first)   # physical first-layer distance
    centres, pdf = analysis.y1plus_pdf(s)
    m = np.mean(s)
    z = (s - m) / (np.std(s) if np.std(s) > 0 else 1.0)
    return {
        "case": case.name, "grid": [case.nx, case.ny, case.nz], "re_tau": case.re_tau,
        "wall": workload.WALL_NAMES[case.wall], "y1_wall_law": case.y1, "tau0": case.tau,
        "eps_uplus": eps, "loglaw_b": b,
        "u_tau_theory": case.u_tau, "u_tau_measured": u_tau_meas,
        "first_layer": {"yplus": float(yplus[0]), "uplus": float(uplus[0])},
        "y1plus": {"mean": float(m), "std": float(np.std(s)), "skew": float(np.mean(z ** 3)),
                   "pdf_peak_at": float(centres[int(np.argmax(pdf))])},
        "profile": {"yplus": [float(v) for v in yplus], "uplus": [float(v) for v in uplus]},
        "run": run_info,
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--case", default="A20", choices=sorted(TABLE1))
    ap.add_argument("--wall", default="wfb", choices=sorted(WALLS))
    ap.add_argument("--y1", type=float, default=1.0, help="wall distance of the wall law (WFB)")
    ap.add_argument("--law", type=int, default=0, help="0 Spalding, 1 log law, 2 power law")
    ap.add_argument("--t-spin", type=float, default=20.0, help="spin-up, in T = D / u_tau")
    ap.add_argument("--t-end", type=float, default=92.0, help="end of the sampling window, in T")
    ap.add_argument("--samples-per-t", type=float, default=10.0)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--a-plus", type=float, default=A_PLUS,
                    help="van Driest constant A+ (0: no damping of the Smagorinsky length)")
    ap.add_argument("--no-profile", action="store_true", help="omit the profile arrays")
    args = ap.parse_args(argv)
    case = table1_case(args.case, args.wall, args.y1, args.seed, args.law)
    out = run(case, args.t_spin, args.t_end, args.samples_per_t, a_plus=args.a_plus)
    out["a_plus"] = args.a_plus
    if args.no_profile:
        out.pop("profile")
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
