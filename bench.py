"""Throughput of the fused WFB LBM-LES channel step on GB300 (MLUPS).

One step = one pass of the whole hot path (gather/stream, moments, BGK +
Smagorinsky + Guo force, WFB wall layers with the Spalding Newton solve,
store) over every cell of the channel. The headline line is the FP32 channel
256 x 64 x 128 (Re_tau 640, WFB walls, seeded log-law + 10% noise); extra
variants (larger grid, FP16-shifted storage) are reported in the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs an independent replica on its own GPU
(replicas only: the channels share nothing); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_04352_gb300 import workload  # noqa: E402

METRIC = "MLUPS and % of HBM roofline, FP32 vs FP16-storage vs batched, at stated err"
BYTES_PER_LUP = {0: 152, 1: 76}     # 19 reads + 19 writes, FP32 / FP16 storage
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0      # GB300 HBM3e nominal, for the second fraction

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture of the current kernel build, keyed by
# (workload, storage, layout); the captures are summarised under profiles/.
# Absent keys report null.
NCU_TRAFFIC = {("c2", "fp32", "pull"): 264.6e6,
               # mean of the even and the odd AA step launch
               ("c3", "fp16", "aa"): 1280.0e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--layout", default="pull", choices=["pull", "aa"],
                    help="two-lattice pull (default) or the single-lattice AA layout")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def headline_kernel(case, precision, layout=0):
    """Step kernel the library selects for this grid and storage (its AUTO
    rule): the four-cell form for FP16 with nx % 4 == 0, else the two-cell form
    for even nx, else the one-cell form; the _aa entries for the AA layout."""
    from paper_2009_04352_gb300 import lbm
    if precision == lbm.FP16_SHIFTED and case.nx % 4 == 0:
        k = "k_step_quad"
    else:
        k = "k_step_pair" if case.nx % 2 == 0 else "k_step"
    return k + "_aa" if layout == lbm.AA else k


def launches_per_step(case, precision, layout=0):
    """Step-kernel launches per step: the two-lattice FP16 four-cell form runs
    an interior-row launch and a wall-row launch; every other form one."""
    from paper_2009_04352_gb300 import lbm
    quad = precision == lbm.FP16_SHIFTED and case.nx % 4 == 0
    return 2 if quad and layout == lbm.PULL2 and case.ny > 2 else 1


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    if isinstance(v, dict):
                        v = v.get("value", v.get("gbs"))
                    return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def whole_job_rate(local_cells, steps, local_ms, dist=None, device="cpu"):
    """Whole-job throughput of N replicas: the cells of all ranks times the
    steps, over the slowest rank's time. Returns (MLUPS, max ms, total cells)."""
    import torch
    if dist is None or not dist.is_initialized():
        return local_cells * steps / (local_ms * 1e-3) / 1e6, local_ms, local_cells
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(local_cells)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ms, cells = float(t.item()), int(c.item())
    return cells * steps / (ms * 1e-3) / 1e6, ms, cells


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def time_channel(case, precision, steps, warmup, stream, clocks=None, mrt=False, layout=0):
    """Device time of `steps` steps (CUDA events on the handle's stream). With
    mrt the paper's LES operator runs: MRT collision, Smagorinsky with van
    Driest damping (A+ = 26, reference u_tau of the case). layout 1 is the
    single-lattice AA layout."""
    import torch
    from paper_2009_04352_gb300 import lbm

    with torch.cuda.stream(stream):
        ch = lbm.Channel.from_case(case, precision=precision, stream=stream.cuda_stream, layout=layout)
        if mrt:
            ch.set_les(lbm.COLLISION_MRT, case.u_tau, 26.0)
        ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
        ch.step(warmup)
        ch.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ctx = clocks if clocks is not None else _Null()
        with ctx:
            ev0.record(stream)
            ch.step(steps)
            ev1.record(stream)
            ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        cons = ch.conservation()
        finite = bool(np.all(np.isfinite(cons)))
        ch.close()
    return ms, finite


def time_batch(precision, steps, stream, peak):
    """The 64-channel ensemble (uneven sizes and Re_tau), one launch per step,
    launch shape from the autotuner."""
    import torch
    from paper_2009_04352_gb300 import autotune, lbm

    cases = workload.batch_cases(64, seed=5)
    with torch.cuda.stream(stream):
        b = lbm.Batch(cases, precision=precision, stream=stream.cuda_stream)
        tuned = autotune.tune_batch(b, steps=3)
        for m, c in zip(b.members, cases):
            m.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
        b.step(5)
        b.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        finite = all(bool(np.all(np.isfinite(m.conservation()))) for m in b.members[:4])
        cells = b.cells
        cfg = b.config()
        b.close()
    gbs = BYTES_PER_LUP[precision] * cells / (ms * 1e-3) / 1e9
    return {"workload": "64 channels, ny in {32,48,64,96,128}, nx=4ny, nz=2ny, Re_tau in {180..2003}",
            "cells": cells, "MLUPS": cells / (ms * 1e-3) / 1e6, "ms_per_step": ms, "GBs": gbs, "frac": gbs / peak,
            "finite": finite, "launch": {"threads": cfg["threads"], "ctas_per_sm": cfg["ctas_per_sm"],
                                         "grid": cfg["grid"], "tiles": cfg["tiles"],
                                         "from_cache": tuned["cached"]}}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def e2e_channel(case, precision, steps, stream, layout=0):
    """Same metric end to end through the public API with host buffers: upload
    the initial field from pinned host memory, run the steps with plane
    statistics sampled every 10 steps, read the moments and statistics back."""
    import torch
    from paper_2009_04352_gb300 import lbm

    f0 = workload_initial_populations(case)
    pinned = torch.from_numpy(f0).pin_memory()
    host_f = pinned.numpy()
    rho = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory().numpy()
    u = torch.empty((3, case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory().numpy()
    with torch.cuda.stream(stream):
        ch = lbm.Channel.from_case(case, precision=precision, stream=stream.cuda_stream, layout=layout)
        ch.set_populations(host_f)      # warm the staging path once
        ch.step(10)
        ch.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch.set_populations(host_f)
        ch.set_stats_every(10)
        ch.step(steps)
        lbm.lbm_moments(ch.handle, rho.ctypes.data, u.ctypes.data, 0)
        st, w, ns = ch.plane_stats()
        t1 = time.perf_counter()
        ch.close()
    h2d = f0.nbytes
    d2h = rho.nbytes + u.nbytes + st.nbytes + w.nbytes
    return (t1 - t0) * 1e3, h2d, d2h


def workload_initial_populations(case):
    """Initial populations f = f^eq(1, u0) of the seeded channel, generated on
    the device by the library and copied back once (outside any timed region)."""
    from paper_2009_04352_gb300 import lbm
    ch = lbm.Channel.from_case(case, stream=0)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    f = ch.populations()
    ch.close()
    return f


def cpu_baseline(case, budget_s=12.0):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the
    workload. Returns the baseline record and the oracle's velocity field after
    the sampled steps, with their count, so that the GPU error can be stated on
    the same workload."""
    import oracle
    L = oracle.Lattice.from_case(case)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    t0 = time.perf_counter()
    L.step(1)
    one = time.perf_counter() - t0
    n = max(1, int(budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    L.step(n)
    dt = time.perf_counter() - t0
    _, u = L.moments()
    L.close()
    rec = {"value": case.cells * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"FP64 oracle, {case.nx}x{case.ny}x{case.nz} WFB channel, {n} steps "
                     f"after 1 warm-up step ({dt:.1f} s)"}
    # the same oracle with its planes spread over all host cores (OpenMP)
    L = oracle.Lattice.from_case(case)
    threads = L.set_threads(os.cpu_count() or 1)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    t0 = time.perf_counter()
    L.step(1)
    one = time.perf_counter() - t0
    m = max(1, int(0.5 * budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    L.step(m)
    dtm = time.perf_counter() - t0
    L.close()
    rec["all_cores"] = {"value": case.cells * m / dtm / 1e6, "unit": "MLUPS", "cores": threads,
                        "sample": f"same oracle, planes in parallel over {threads} threads, {m} steps ({dtm:.1f} s)"}
    return rec, u, n + 1


def stated_error(case, u_ref, steps, stream):
    """Relative L_inf of the GPU velocity against the FP64 oracle after the same
    steps from the same seeded field, FP32 and FP16 storage."""
    import torch
    from paper_2009_04352_gb300 import lbm
    out = {}
    for name, prec in (("fp32", lbm.FP32), ("fp16", lbm.FP16_SHIFTED)):
        with torch.cuda.stream(stream):
            ch = lbm.Channel.from_case(case, precision=prec, stream=stream.cuda_stream)
            ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
            ch.step(steps)
            _, u = ch.moments()
            ch.close()
        out[name] = float(np.max(np.abs(u - u_ref)) / np.max(np.abs(u_ref)))
    return {"rel_linf_u": out, "steps": steps, "bound": {"fp32": 1e-5, "fp16": 5e-3},
            "vs": "FP64 oracle, same seeded field, same workload"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def main_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    case = workload.CASES[args.workload]
    import oracle
    L = oracle.Lattice.from_case(case)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    # each "step" of this arm is a bounded sample: one oracle step of the workload
    L.step(max(0, min(args.warmup, 1)))
    steps = max(1, min(args.steps, 8))
    t0 = time.perf_counter()
    L.step(steps)
    dt = time.perf_counter() - t0
    L.close()
    val = case.cells * steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": dt * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": case.name, "cells": case.cells},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 oracle, {steps} steps of {case.name} (cpu: {cpu_model()})"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return main_reference(args)

    import torch
    import __graft_entry__
    __graft_entry__.build()

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2009_04352_gb300 import lbm

    precision = lbm.FP32 if args.precision == "fp32" else lbm.FP16_SHIFTED
    case = workload.CASES[args.workload]
    stream = torch.cuda.Stream()
    peak, peak_src = measured_peaks()

    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    layout = lbm.AA if args.layout == "aa" else lbm.PULL2
    ms, finite = time_channel(case, precision, args.steps, args.warmup, stream, clocks, layout=layout)
    torch.cuda.synchronize()
    per_gpu_mlups = case.cells * args.steps / (ms * 1e-3) / 1e6
    mlups, ms, total_cells = whole_job_rate(case.cells, args.steps, ms, pg, "cuda")
    if pg:
        pg.barrier()
    kernel_ms = ms / args.steps
    achieved = BYTES_PER_LUP[precision] * case.cells / (kernel_ms * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        e2e_steps = min(args.steps, 2000)
        e_ms, h2d, d2h = e2e_channel(case, precision, e2e_steps, stream, layout)
        e_val, e_ms, _ = whole_job_rate(case.cells, e2e_steps, e_ms, pg, "cuda")
        e2e = {"value": e_val, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
               "steps": e2e_steps,
               "what": "C-ABI with host buffers: pinned FP64 initial field uploaded, steps with "
                       "plane statistics every 10 steps, moments and statistics read back"}

    variants = {}
    if not args.no_variants and rank == 0:
        for name, prec in (("c5_batch64_fp32", lbm.FP32), ("c5_batch64_fp16", lbm.FP16_SHIFTED)):
            variants[name] = time_batch(prec, 30, stream, peak)
    if not args.no_variants and rank == 0:
        for name, wl, prec, steps, mrt in (("c3_fp32", "c3", lbm.FP32, 2000, False),
                                           ("c3_fp16", "c3", lbm.FP16_SHIFTED, 2000, False),
                                           ("c4_fp32", "c4", lbm.FP32, 300, False),
                                           ("c4_fp16", "c4", lbm.FP16_SHIFTED, 300, False),
                                           ("c3_mrt_vandriest_fp32", "c3", lbm.FP32, 1000, True),
                                           ("c3_mrt_vandriest_fp16", "c3", lbm.FP16_SHIFTED, 1000, True),
                                           ("c3_loglaw_fp32", "c3+log", lbm.FP32, 1000, False),
                                           ("c3_powerlaw_fp32", "c3+power", lbm.FP32, 1000, False),
                                           ("c3_aa_fp32", "c3+aa", lbm.FP32, 2000, False),
                                           ("c3_aa_fp16", "c3+aa", lbm.FP16_SHIFTED, 2000, False),
                                           ("c4_aa_fp32", "c4+aa", lbm.FP32, 300, False),
                                           ("c4_aa_fp16", "c4+aa", lbm.FP16_SHIFTED, 300, False)):
            wl, *opts = wl.split("+")
            c = workload.CASES[wl]
            if "log" in opts:
                c = c.with_(wall_law=lbm.LAW_LOG)
            if "power" in opts:
                c = c.with_(wall_law=lbm.LAW_POWER)
            vlayout = lbm.AA if "aa" in opts else lbm.PULL2
            vms, vfin = time_channel(c, prec, steps, 20, stream, mrt=mrt, layout=vlayout)
            kms = vms / steps
            gbs = BYTES_PER_LUP[prec] * c.cells / (kms * 1e-3) / 1e9
            variants[name] = {"workload": c.name, "cells": c.cells, "MLUPS": c.cells * steps / (vms * 1e-3) / 1e6,
                              "ms_per_step": kms, "GBs": gbs, "frac": gbs / peak, "finite": vfin}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": kernel_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == lbm.FP32 else "f32 (fp16 storage)",
        "data": "synthetic",
        "config": {"workload": case.name, "grid": [case.nx, case.ny, case.nz], "cells": case.cells,
                   "re_tau": case.re_tau, "tau0": case.tau, "C_s": case.cs, "wall": "wfb",
                   "storage": args.precision,
                   "layout": "single-lattice AA" if layout == lbm.AA else "two-lattice pull",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (129 MB): %s %.0f MB lattice%s per step" % (
                       "one" if layout == lbm.AA else "two", BYTES_PER_LUP[precision] / 2 * case.cells / 1e6,
                       "" if layout == lbm.AA else "s")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((args.workload, args.precision, args.layout)),
                     "peak_source": peak_src, "kernel": headline_kernel(case, precision, layout),
                     "bytes_per_lup": BYTES_PER_LUP[precision],
                     "frac_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS},
        "per_gpu_MLUPS": per_gpu_mlups, "finite": finite,
        "gpu_launches": args.steps * launches_per_step(case, precision, layout),
        "clocks": clocks.summary(),
    }
    if e2e:
        line["e2e"] = e2e
    if variants:
        line["variants"] = variants
    if world == 1 and not args.no_cpu_baseline:
        rec, u_ref, n_ref = cpu_baseline(case)
        rec["cpu"] = cpu_model()
        line["cpu_baseline"] = rec
        line["err_vs_fp64"] = stated_error(case, u_ref, n_ref, stream)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
