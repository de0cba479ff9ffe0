"""Write <case>_storage_floor.txt: the storage-rounding floor of a channel
against the FP64 oracle over its first 100 steps.

The GPU stores every population as a deviation f_a - w_a in FP32 or FP16,
rounded to nearest once per step. Running the oracle with the same rounding
applied to its state after the initial field and after every step (here, in
the script: the oracle itself stays plain FP64) gives the error that storage
alone causes. For each checkpoint and storage precision the file lists the
relative L_inf of that rounded run against the plain oracle for
  u          velocity (Eq. 2 with the Guo half-force shift),
  rho_out    density deviation rho - 1, with rho rounded to FP32 as the
             library's moments return it,
  f_minus_w  population deviations,
  tau_w      wall stress (Eqs. 15-17).
Only the oracle and numpy run here.

    python tests/golden/make_storage_floor.py [--case c3] [--threads N]
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

CHECKPOINTS = (1, 10, 100)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None, None, None]


def round_state(L, dtype):
    f = L.populations()
    f -= W
    f[...] = f.astype(dtype)
    f += W
    L.set_populations(f)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="c3")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    case = workload.CASES[args.case]
    t0 = time.time()
    ref = oracle.Lattice.from_case(case)
    ref.set_threads(args.threads)
    ref.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    runs = {}
    for name, dt in (("fp32", np.float32), ("fp16", np.float16)):
        L = oracle.Lattice.from_case(case)
        L.set_threads(args.threads)
        L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
        round_state(L, dt)
        runs[name] = (L, dt)
    rows = []
    for t in range(1, CHECKPOINTS[-1] + 1):
        ref.step(1)
        for L, dt in runs.values():
            L.step(1)
            round_state(L, dt)
        if t in CHECKPOINTS:
            rho_r, u_r = ref.moments()
            tw_r = ref.wall_stress()
            f_r = ref.populations() - W
            for name, (L, _) in runs.items():
                rho, u = L.moments()
                rho32 = rho.astype(np.float32).astype(np.float64)
                f = L.populations() - W
                rows.append((name, t, rel(u, u_r), rel(rho32 - 1.0, rho_r - 1.0), rel(f, f_r),
                             rel(L.wall_stress(), tw_r)))
                del f
            del f_r
            print(f"step {t} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, f"{args.case}_storage_floor.txt"), "w") as fh:
        fh.write(f"# {case.name}: storage-rounding floor against the FP64 oracle (relative L_inf)\n")
        fh.write(f"# written by: python tests/golden/make_storage_floor.py --case {args.case} "
                 f"--threads {args.threads} ({time.time() - t0:.0f} s)\n")
        fh.write("# storage step u rho_out f_minus_w tau_w\n")
        for r in rows:
            fh.write("%s %d %.6e %.6e %.6e %.6e\n" % r)


if __name__ == "__main__":
    main()
