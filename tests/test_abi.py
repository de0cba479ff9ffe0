"""Host-side checks of the C ABI: the library builds, loads without a GPU,
exports every entry point declared in include/lbm.h, and rejects invalid
arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(lbm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2009_04352_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("lbm_create", "lbm_step", "lbm_moments", "lbm_wall_stress", "lbm_plane_stats",
                     "lbm_populations", "lbm_destroy", "lbm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(built_lib):
    for name in _declared():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_symbol():
    from paper_2009_04352_gb300 import lbm
    assert set(_declared()) <= set(lbm.exported_symbols())


def test_invalid_arguments_rejected_without_device():
    from paper_2009_04352_gb300 import lbm
    bad = [dict(nx=8, ny=1, nz=8, tau=0.6),            # ny < 2
           dict(nx=0, ny=8, nz=8, tau=0.6),            # empty grid
           dict(nx=8, ny=8, nz=8, tau=0.5),            # tau must exceed 1/2
           dict(nx=8, ny=8, nz=8, tau=0.6, cs=-1.0),   # negative C_s
           dict(nx=8, ny=8, nz=8, tau=0.6, wall=7),    # unknown wall
           dict(nx=8, ny=8, nz=8, tau=0.6, precision=5),
           dict(nx=8, ny=8, nz=8, tau=0.6, layout=3),
           dict(nx=1 << 16, ny=1 << 10, nz=1 << 10, tau=0.6),  # > 2^31 cells
           dict(nx=8, ny=8, nz=8, tau=0.6, law=3),     # unknown wall law
           dict(nx=8, ny=8, nz=8, tau=0.6, law=lbm.LAW_LOG, B=0.2),  # log branches never cross
           # corrupted configurations: NaN relaxation time or Smagorinsky
           # constant, non-finite body force
           dict(nx=8, ny=8, nz=8, tau=float("nan")),
           dict(nx=8, ny=8, nz=8, tau=0.6, cs=float("nan")),
           dict(nx=8, ny=8, nz=8, tau=0.6, force=(float("inf"), 0, 0)),
           dict(nx=8, ny=8, nz=8, tau=0.6, force=(0, float("nan"), 0))]
    for kw in bad:
        kw = dict(kw)
        args = dict(cs=0.1, force=(1e-6, 0, 0), wall=lbm.WALL_WFB, precision=lbm.FP32, layout=lbm.PULL2,
                    law=lbm.LAW_SPALDING, B=5.5)
        args.update(kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create(args.pop("nx"), args.pop("ny"), args.pop("nz"), args.pop("tau"), args.pop("cs"),
                           args.pop("force"), wall=args["wall"], B=args["B"], precision=args["precision"],
                           layout=args["layout"], stream=0, law=args["law"])
        assert ei.value.code == lbm.LBM_ERR_ARG
        assert lbm.lib().lbm_last_error().decode()


def test_null_handle_calls_fail_cleanly():
    from paper_2009_04352_gb300 import lbm
    L = lbm.lib()
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert L.lbm_sync(None) == lbm.LBM_ERR_ARG
    assert L.lbm_set_wait_limit(None, 1) == lbm.LBM_ERR_ARG
    assert L.lbm_get_step(None) == -1
    L.lbm_destroy(None)


def test_population_bytes_host_arithmetic():
    from paper_2009_04352_gb300 import lbm
    # rows padded to a multiple of 32 cells, 19 planes
    assert lbm.lbm_population_bytes(64, 32, 32, lbm.FP32) == 19 * 64 * 32 * 32 * 4
    assert lbm.lbm_population_bytes(37, 6, 5, lbm.FP32) == 19 * 64 * 6 * 5 * 4
    assert lbm.lbm_population_bytes(33, 2, 3, lbm.FP16_SHIFTED) == 19 * 64 * 2 * 3 * 2
    assert lbm.lbm_population_bytes(0, 2, 3, lbm.FP32) == 0
    assert lbm.lbm_population_bytes(8, 8, 8, 7) == 0


def test_create_from_buffers_rejects_bad_buffers_without_device():
    from paper_2009_04352_gb300 import lbm
    bad = [dict(pop0=None, pop1=None, layout=lbm.PULL2),          # no buffer
           dict(pop0=4096, pop1=None, layout=lbm.PULL2),          # two-lattice needs two
           dict(pop0=4096, pop1=8192, layout=lbm.AA),             # AA takes one
           dict(pop0=4104, pop1=8192, layout=lbm.PULL2),          # misaligned
           dict(pop0=4096, pop1=8200, layout=lbm.PULL2)]
    for kw in bad:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create_from_buffers(8, 8, 8, 0.6, 0.1, (1e-6, 0, 0), kw["pop0"], kw["pop1"],
                                        layout=kw["layout"], stream=0)
        assert ei.value.code == lbm.LBM_ERR_ARG


def test_bench_launch_and_kernel_bookkeeping():
    """bench.py's count of step-kernel launches and its name of the selected
    kernel follow the library's selection rules (host logic only)."""
    import bench
    from paper_2009_04352_gb300 import lbm, workload
    c2, c3 = workload.CASES["c2"], workload.CASES["c3"]
    assert bench.launches_per_step(c2, lbm.FP32) == 1
    assert bench.launches_per_step(c3, lbm.FP16_SHIFTED) == 2           # interior + wall rows
    assert bench.launches_per_step(c3, lbm.FP16_SHIFTED, lbm.AA) == 1
    assert bench.launches_per_step(c3, lbm.FP16_SHIFTED, mrt=True) == 1   # one launch, wall tile called
    assert bench.launches_per_step(c3.with_(ny=2), lbm.FP16_SHIFTED) == 1
    node = c3.with_(ny=129, wall=workload.WALL_WFB_NODE)
    assert bench.launches_per_step(node, lbm.FP16_SHIFTED, mrt=True) == 2     # node rows: two-cell wall launch
    assert bench.headline_kernel(c2, lbm.FP32) == "k_step_pair"
    assert bench.headline_kernel(c3, lbm.FP16_SHIFTED) == "k_step_quad"
    assert bench.headline_kernel(c3, lbm.FP16_SHIFTED, lbm.AA) == "k_step_quad_aa"
    assert bench.headline_kernel(c2.with_(nx=37), lbm.FP32) == "k_step"


def test_autotune_rejects_bad_arguments_without_device(built_lib):
    from paper_2009_04352_gb300 import lbm
    assert lbm.lib().lbm_autotune(None, 4, None, None) == lbm.LBM_ERR_ARG
