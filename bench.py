"""Throughput of the fused WFB LBM-LES channel step on GB300 (MLUPS).

One step = one pass of the whole hot path (gather/stream, moments, BGK +
Smagorinsky + Guo force, WFB wall layers with the Spalding Newton solve,
store) over every cell of the channel. The headline line is the large-grid
roofline channel 1024 x 256 x 512 (134M cells, Re_tau 2003, WFB walls, seeded
log-law + 10% noise) with FP32 two-lattice storage; the FP16-storage AA single
lattice of the same grid, the other grids, the paper's MRT + van Driest LES
operator, the other wall functions and the batched ensemble are reported as
variants in the same line (the ensemble last).

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
GRAPH_STEPS = 16              # steps per replayed CUDA graph in the library
SAMPLE_CELLS = 2_100_000      # cells of the bounded oracle sample (a z-slab of the workload)

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture of the current kernel build, keyed by
# (workload, storage, layout, collision); the captures are summarised under
# profiles/. A workload too large for a multi-metric capture is captured as a
# z-slab of the same channel and scaled by its cell count (traffic per cell
# does not depend on nz). Absent keys report null.
NCU_TRAFFIC = {
    # k_step_pair<float>, 1024x256x16 slab: 597.5 MB per launch (142.5 B/cell) x 32
    ("c4", "fp32", "pull", "bgk"): 19.121e9,
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c4", choices=["c1", "c2", "c3", "c4"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--layout", default="pull", choices=["pull", "aa"],
                    help="two-lattice pull (default) or the single-lattice AA layout")
    ap.add_argument("--les", default="bgk", choices=["bgk", "mrt"],
                    help="collision of the timed channel: BGK + Smagorinsky (default) or the paper's MRT + "
                         "Smagorinsky + van Driest (A+ = 26)")
    ap.add_argument("--nz", type=int, default=0,
                    help="run a z-slab of the workload with this many planes (same nx, ny and parameters), "
                         "for bounded profiler captures; 0 runs the whole grid")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args(argv)


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


def launches_per_step(case, precision, layout=0, mrt=False):
    """Step-kernel launches per step: the two-lattice FP16 four-cell form with
    BGK, or with wall nodes, runs an interior-row launch and a wall-row launch
    (with MRT and halfway walls one launch whose wall-row CTAs call a
    separately compiled tile); every other form one."""
    from paper_2009_04352_gb300 import lbm
    quad = precision == lbm.FP16_SHIFTED and case.nx % 4 == 0
    node = case.wall == workload.WALL_WFB_NODE
    return 2 if quad and layout == lbm.PULL2 and (not mrt or node) and case.ny > 2 else 1


def sample_case(case, cells=SAMPLE_CELLS):
    """Bounded sample of a workload for the CPU oracle: a z-slab of the same
    channel (same nx, ny and lattice parameters, periodic in z) of about
    `cells` cells; the workload itself if it is that small."""
    if case.cells <= cells:
        return case
    nz = max(2, cells // (case.nx * case.ny))
    return case.with_(nz=nz, name=f"{case.name}_zslab{nz}")


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
    """nvidia-smi clocks, utilisation and throttle reasons every 50 ms for the
    whole run, each sample stamped with the host clock so that the samples of
    one timed region can be picked out."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append((time.perf_counter(), parts))

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _num(s):
        try:
            return float(s)
        except ValueError:
            return None

    def summary(self, t0=None, t1=None):
        """Median SM clock of the samples in [t0, t1] (all samples if no bounds),
        the maximum clock, and every throttle reason seen. Without a sample in
        the window the summary falls back to the samples of the whole run taken
        under load (utilisation >= 50%) and says so."""
        rows = [p for t, p in self.rows if (t0 is None or t >= t0) and (t1 is None or t <= t1)]
        window = "timed region" if t0 is not None else "whole run"
        if not rows:
            rows = [p for _, p in self.rows if (self._num(p[3]) or 0.0) >= 50.0]
            window = "whole run, samples under load (none fell in the timed region)"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [v for v in (self._num(p[0]) for p in rows) if v is not None]
        mx = [v for v in (self._num(p[1]) for p in rows) if v is not None]
        reasons = sorted({self.REASONS[i] for p in rows for i in range(4) if p[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


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


def time_channel(case, precision, steps, warmup, stream, mrt=False, layout=0, barrier=None):
    """Device time of `steps` steps (CUDA events on the handle's stream) after
    `warmup` untimed steps; the library builds its step graphs on the first
    step call, inside the warm-up. With mrt the paper's LES operator runs: MRT
    collision, Smagorinsky with van Driest damping (A+ = 26, reference u_tau of
    the case). layout 1 is the single-lattice AA layout. Returns (ms, finite,
    host-clock bounds of the timed region)."""
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
        if barrier:
            barrier()
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        ev0.record(stream)
        ch.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        h1 = time.perf_counter()
        ms = ev0.elapsed_time(ev1)
        cons = ch.conservation()
        finite = bool(np.all(np.isfinite(cons)))
        ch.close()
    return ms, finite, (h0, h1)


def time_batch(precision, steps, stream, peak, clocks):
    """The 64-channel ensemble (uneven sizes and Re_tau), one launch per step,
    launch shape from the autotuner."""
    import torch
    from paper_2009_04352_gb300 import autotune, lbm

    cases = workload.batch_cases(64, seed=5)
    with torch.cuda.stream(stream):
        b = lbm.Batch(cases, precision=precision, stream=stream.cuda_stream)
        # one graph chunk per candidate, so that every form is timed as it runs
        tuned = autotune.tune_batch(b, steps=GRAPH_STEPS)
        for m, c in zip(b.members, cases):
            m.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
        b.step(2 * GRAPH_STEPS)
        b.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        ev0.record(stream)
        b.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        h1 = time.perf_counter()
        ms = ev0.elapsed_time(ev1) / steps
        finite = all(bool(np.all(np.isfinite(m.conservation()))) for m in b.members[:4])
        cells = b.cells
        cfg = b.config()
        b.close()
    gbs = BYTES_PER_LUP[precision] * cells / (ms * 1e-3) / 1e9
    return {"workload": "64 channels, ny in {32,48,64,96,128}, nx=4ny, nz=2ny, Re_tau in {180..2003}",
            "cells": cells, "MLUPS": cells / (ms * 1e-3) / 1e6, "ms_per_step": ms, "GBs": gbs, "frac": gbs / peak,
            "finite": finite, "sm_mhz": clocks.summary(h0, h1)["sm_mhz"],
            "launch": {"form": "persistent" if cfg["form"] == lbm.BATCH_PERSISTENT else "member grids",
                       "threads": cfg["threads"], "ctas_per_sm": cfg["ctas_per_sm"], "streams": cfg["streams"],
                       "from_cache": tuned["cached"]}}


def e2e_channel(case, precision, steps, stream, layout=0):
    """Same metric end to end through the public API with host buffers: upload
    the initial populations (FP64, pinned host memory), run the steps with
    plane statistics sampled every 10 steps, read the moments and statistics
    back, all inside the wall-clock region."""
    import torch
    from paper_2009_04352_gb300 import lbm

    host_f = torch.empty((19, case.nz, case.ny, case.nx), dtype=torch.float64, pin_memory=True).numpy()
    workload_initial_populations(case, host_f)
    rho = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory().numpy()
    u = torch.empty((3, case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory().numpy()
    with torch.cuda.stream(stream):
        ch = lbm.Channel.from_case(case, precision=precision, stream=stream.cuda_stream, layout=layout)
        ch.set_populations(host_f)      # warm the staging path once
        ch.step(2 * GRAPH_STEPS)
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
    h2d = host_f.nbytes
    d2h = rho.nbytes + u.nbytes + st.nbytes + w.nbytes
    del host_f
    return (t1 - t0) * 1e3, h2d, d2h


def workload_initial_populations(case, out):
    """Initial populations f = f^eq(1, u0) of the seeded channel, generated on
    the device by the library and copied once into `out` (outside any timed
    region)."""
    from paper_2009_04352_gb300 import lbm
    ch = lbm.Channel.from_case(case, stream=0)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    lbm.lbm_populations(ch.handle, out)
    ch.close()
    return out


def cpu_baseline(case, budget_s=12.0):
    """The FP64 oracle as it stands on a bounded sample of the workload (a
    z-slab of the same channel), single-threaded and on all host cores."""
    import oracle
    s = sample_case(case)
    L = oracle.Lattice.from_case(s)
    L.init_channel(workload.u_mean_profile(s), workload.noise_amplitude(s), s.seed)
    t0 = time.perf_counter()
    L.step(1)
    one = time.perf_counter() - t0
    n = max(1, int(budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    L.step(n)
    dt = time.perf_counter() - t0
    L.close()
    rec = {"value": s.cells * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"FP64 oracle, {s.nx}x{s.ny}x{s.nz} z-slab of the {case.nx}x{case.ny}x{case.nz} WFB channel "
                     f"(same parameters), {n} steps after 1 warm-up step ({dt:.1f} s)"}
    L = oracle.Lattice.from_case(s)
    threads = L.set_threads(os.cpu_count() or 1)
    L.init_channel(workload.u_mean_profile(s), workload.noise_amplitude(s), s.seed)
    t0 = time.perf_counter()
    L.step(1)
    one = time.perf_counter() - t0
    m = max(1, int(0.5 * budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    L.step(m)
    dtm = time.perf_counter() - t0
    L.close()
    rec["all_cores"] = {"value": s.cells * m / dtm / 1e6, "unit": "MLUPS", "cores": threads,
                        "sample": f"same oracle and slab, planes in parallel over {threads} threads, {m} steps "
                                  f"({dtm:.1f} s)"}
    return rec


def stated_error(case, stream, steps=100):
    """Relative L_inf against the FP64 oracle after `steps` steps from the same
    seeded field, on the z-slab sample of the workload (same kernel form and
    launch shape per row), FP32 and FP16 storage: velocity, density deviation,
    population deviations f - w, wall stress."""
    import torch
    import oracle
    from paper_2009_04352_gb300 import lbm
    s = sample_case(case)
    W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None, None, None]
    L = oracle.Lattice.from_case(s)
    L.set_threads(os.cpu_count() or 1)
    L.init_channel(workload.u_mean_profile(s), workload.noise_amplitude(s), s.seed)
    L.step(steps)
    rho_o, u_o = L.moments()
    f_o = L.populations() - W
    tw_o = L.wall_stress()
    L.close()

    def rel(a, b):
        return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))

    out = {}
    for name, prec in (("fp32", lbm.FP32), ("fp16", lbm.FP16_SHIFTED)):
        with torch.cuda.stream(stream):
            ch = lbm.Channel.from_case(s, precision=prec, stream=stream.cuda_stream)
            ch.init_channel(workload.u_mean_profile(s), workload.noise_amplitude(s), s.seed)
            ch.step(steps)
            rho, u = ch.moments()
            f = ch.populations() - W
            out[name] = {"u": rel(u, u_o), "rho_minus_1": rel(rho - 1.0, rho_o - 1.0), "f_minus_w": rel(f, f_o),
                         "tau_w": rel(ch.wall_stress(), tw_o)}
            ch.close()
    return {"rel_linf": out, "steps": steps, "bound": {"fp32": 1e-5, "fp16": 5e-3},
            "vs": f"FP64 oracle, same seeded field, {s.nx}x{s.ny}x{s.nz} z-slab of the workload"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def line_config(case, args, world):
    """The workload of the line (the same dict for both arms)."""
    aa = args.layout == "aa"
    return {"workload": case.name, "grid": [case.nx, case.ny, case.nz], "cells": case.cells,
            "re_tau": case.re_tau, "tau0": case.tau, "C_s": case.cs, "wall": "wfb",
            "storage": args.precision, "les": "MRT + van Driest" if args.les == "mrt" else "BGK",
            "layout": "single-lattice AA" if aa else "two-lattice pull",
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (129 MB): %s %.0f MB lattice%s per step" % (
                "one" if aa else "two", BYTES_PER_LUP[0 if args.precision == "fp32" else 1] / 2 * case.cells / 1e6,
                "" if aa else "s")}


def main_reference(args):
    """The oracle on the host cores, each step a bounded sample of the
    workload (one oracle step of its z-slab)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    case = workload.CASES[args.workload]
    if args.nz > 0:
        case = case.with_(nz=args.nz, name=f"{case.name}_zslab{args.nz}")
    s = sample_case(case)
    import oracle
    L = oracle.Lattice.from_case(s)
    threads = L.set_threads(os.cpu_count() or 1)
    if args.les == "mrt":
        L.set_les(1, case.u_tau, 26.0)
    L.init_channel(workload.u_mean_profile(s), workload.noise_amplitude(s), s.seed)
    L.step(max(0, args.warmup))
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    L.step(steps)
    dt = time.perf_counter() - t0
    L.close()
    val = s.cells * steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": line_config(case, args, world),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"FP64 oracle, each step one step of the {s.nx}x{s.ny}x{s.nz} z-slab of "
                                       f"{case.name} over {threads} threads (cpu: {cpu_model()})"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


VARIANTS = (  # name, workload[+options], storage, steps
    ("c2_fp32", "c2", 0, 2000),
    ("c3_fp32", "c3", 0, 1000),
    ("c3_fp16", "c3", 1, 1000),
    ("c4_fp16", "c4", 1, 200),
    ("c4_aa_fp32", "c4+aa", 0, 200),
    ("c4_aa_fp16", "c4+aa", 1, 200),
    ("c3_aa_fp32", "c3+aa", 0, 1000),
    ("c3_aa_fp16", "c3+aa", 1, 1000),
    ("c3_mrt_vandriest_fp32", "c3+mrt", 0, 1000),
    ("c3_mrt_vandriest_fp16", "c3+mrt", 1, 1000),
    ("c3_loglaw_fp32", "c3+log", 0, 1000),
    ("c3_powerlaw_fp32", "c3+power", 0, 1000),
)


def run_variants(stream, peak, clocks):
    from paper_2009_04352_gb300 import lbm
    out = {}
    for name, spec, prec, steps in VARIANTS:
        wl, *opts = spec.split("+")
        c = workload.CASES[wl]
        if "log" in opts:
            c = c.with_(wall_law=lbm.LAW_LOG)
        if "power" in opts:
            c = c.with_(wall_law=lbm.LAW_POWER)
        layout = lbm.AA if "aa" in opts else lbm.PULL2
        ms, fin, (h0, h1) = time_channel(c, prec, steps, 2 * GRAPH_STEPS, stream, mrt="mrt" in opts, layout=layout)
        kms = ms / steps
        gbs = BYTES_PER_LUP[prec] * c.cells / (kms * 1e-3) / 1e9
        out[name] = {"workload": c.name, "cells": c.cells, "MLUPS": c.cells * steps / (ms * 1e-3) / 1e6,
                     "ms_per_step": kms, "GBs": gbs, "frac": gbs / peak, "finite": fin,
                     "sm_mhz": clocks.summary(h0, h1)["sm_mhz"]}
    for name, prec in (("c5_batch64_fp32", lbm.FP32), ("c5_batch64_fp16", lbm.FP16_SHIFTED)):
        out[name] = time_batch(prec, 100, stream, peak, clocks)
    return out


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
    layout = lbm.AA if args.layout == "aa" else lbm.PULL2
    case = workload.CASES[args.workload]
    if args.nz > 0:
        case = case.with_(nz=args.nz, name=f"{case.name}_zslab{args.nz}")
    stream = torch.cuda.Stream()
    peak, peak_src = measured_peaks()

    with ClockSampler(local) as clocks:
        ms, finite, (h0, h1) = time_channel(case, precision, args.steps, args.warmup, stream, layout=layout,
                                            mrt=args.les == "mrt", barrier=pg.barrier if pg else None)
        torch.cuda.synchronize()
        per_gpu_mlups = case.cells * args.steps / (ms * 1e-3) / 1e6
        mlups, ms, total_cells = whole_job_rate(case.cells, args.steps, ms, pg, "cuda")
        if pg:
            pg.barrier()
        kernel_ms = ms / args.steps
        achieved = BYTES_PER_LUP[precision] * case.cells / (kernel_ms * 1e-3) / 1e9

        e2e = None
        if not args.no_e2e:
            e_ms, h2d, d2h = e2e_channel(case, precision, args.steps, stream, layout)
            e_val, e_ms, _ = whole_job_rate(case.cells, args.steps, e_ms, pg, "cuda")
            e2e = {"value": e_val, "unit": "MLUPS",
                   "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                   "steps": args.steps,
                   "what": "C-ABI with host buffers: pinned FP64 initial field uploaded, steps with plane "
                           "statistics every 10 steps, moments and statistics read back"}

        extra = {}
        if world == 1 and not args.no_cpu_baseline:
            rec = cpu_baseline(case)
            rec["cpu"] = cpu_model()
            extra["cpu_baseline"] = rec
            extra["err_vs_fp64"] = stated_error(case, stream)
        variants = run_variants(stream, peak, clocks) if (not args.no_variants and rank == 0) else {}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": kernel_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == lbm.FP32 else "f32 (fp16 storage)",
        "data": "synthetic",
        "config": line_config(case, args, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((args.workload, args.precision, args.layout, args.les))
                     if args.nz == 0 else None,
                     "peak_source": peak_src, "kernel": headline_kernel(case, precision, layout),
                     "bytes_per_lup": BYTES_PER_LUP[precision],
                     "frac_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS},
        "per_gpu_MLUPS": per_gpu_mlups, "finite": finite,
        "gpu_launches": args.steps * launches_per_step(case, precision, layout, args.les == "mrt"),
        "clocks": clocks.summary(h0, h1),
        "clocks_whole_run": clocks.summary(),
    }
    if e2e:
        line["e2e"] = e2e
    line.update(extra)
    if variants:
        line["variants"] = variants
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
