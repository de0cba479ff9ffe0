"""Write c2_statistics.txt: time- and plane-averaged statistics of the
256 x 64 x 128 Re_tau 640 channel (WFB walls, seeded log-law + noise field)
from the FP64 oracle, over 40000 steps in four windows of 10000 steps.

The statistics follow the procedure of Sec. 3.1: each wall-normal layer is
averaged in time (samples every 10 steps, taken from the state f(t) at the
start of step t) and over its plane. Per window the file stores the sums over
the samples and the cells of each layer of rho, u_x and u_x^2 (u with the Guo
half-force shift, as the library's moments), and per wall the sums over the
samples and wall cells of tau_w,x and |tau_w| of the step that starts from the
sampled state. The run uses only the oracle (all host cores for the
unsampled steps; the oracle's parallel mode is bitwise its serial result) and
numpy for the plane sums.

    python tests/golden/make_c2_statistics.py [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_04352_gb300 import workload  # noqa: E402

STEPS = 40000
WINDOW = 10000
EVERY = 10
OUT = os.path.join(HERE, "c2_statistics.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--steps", type=int, default=STEPS)
    ap.add_argument("--window", type=int, default=WINDOW)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    case = workload.CASES["c2"]
    L = oracle.Lattice.from_case(case)
    threads = L.set_threads(args.threads)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    nwin = args.steps // args.window
    planes = np.zeros((nwin, case.ny, 3))     # rho, u_x, u_x^2 summed over samples and cells
    walls = np.zeros((nwin, 2, 2))            # tau_w,x and |tau_w| summed over samples and wall cells
    samples = np.zeros(nwin, dtype=np.int64)
    t0 = time.time()
    for t in range(0, args.steps, EVERY):
        w = t // args.window
        rho, u = L.moments()                  # state f(t)
        planes[w, :, 0] += rho.sum(axis=(0, 2))
        planes[w, :, 1] += u[0].sum(axis=(0, 2))
        planes[w, :, 2] += (u[0] * u[0]).sum(axis=(0, 2))
        L.step(1)                             # the sampled step t -> t + 1
        tw = L.wall_stress()                  # its wall stress, from f(t)
        walls[w, :, 0] += tw[..., 0].sum(axis=(1, 2))
        walls[w, :, 1] += np.sqrt(tw[..., 0] ** 2 + tw[..., 1] ** 2).sum(axis=(1, 2))
        samples[w] += 1
        L.step(EVERY - 1)
        if (t // EVERY) % 200 == 0:
            print(f"step {t} ({time.time() - t0:.0f} s)", flush=True)
    L.close()
    with open(args.out, "w") as fh:
        fh.write("# c2 channel 256x64x128, Re_tau 640, WFB (Spalding), seed 2: FP64 oracle statistics\n")
        fh.write(f"# written by: python tests/golden/make_c2_statistics.py --threads {threads} "
                 f"--steps {args.steps} --window {args.window} ({time.time() - t0:.0f} s)\n")
        fh.write(f"# windows of {args.window} steps, samples every {EVERY} steps from the state at the start of the step\n")
        fh.write("# plane rows: window y sum_rho sum_ux sum_ux2 (sums over samples and the nx*nz cells of layer y)\n")
        fh.write("# wall rows: window wall sum_tau_wx sum_abs_tau_w (sums over samples and nx*nz wall cells)\n")
        fh.write(f"cells_per_plane {case.nx * case.nz}\n")
        for w in range(nwin):
            fh.write(f"samples {w} {samples[w]}\n")
        for w in range(nwin):
            for y in range(case.ny):
                fh.write("plane %d %d %.17g %.17g %.17g\n" % (w, y, *planes[w, y]))
        for w in range(nwin):
            for k in range(2):
                fh.write("wall %d %d %.17g %.17g\n" % (w, k, *walls[w, k]))


if __name__ == "__main__":
    main()
