"""Steps launched back to back against steps separated by host synchronisation.

Consecutive step kernels on a stream overlap: most launch with programmatic
dependent launch, so the next step's grid is already resident while the
current one drains, and a CUDA-graph chunk of 16 steps runs them back to back.
A kernel that read the previous step's output before its
griddepcontrol.wait, or through the read-only path while that output was
still being written, would read stale populations only in the overlapped
form. Separated steps (one step per call, the state copied to the host in
between) cannot overlap, so the two must agree bitwise, for every kernel form,
storage precision, layout and wall kind, across graph chunks started from
either phase."""
import numpy as np
import pytest

from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu

CASE = workload.CASES["c1"]
RUNS = (3, 17, 16)            # 3 single launches back to back, then a chunk + 1 from phase 1, a chunk from phase 0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()


def _forms():
    out = []
    for prec in (lbm.FP32, lbm.FP16_SHIFTED):
        kernels = [lbm.KERNEL_CELL, lbm.KERNEL_PAIR] + ([lbm.KERNEL_QUAD] if prec == lbm.FP16_SHIFTED else [])
        for k in kernels:
            for layout in (lbm.PULL2, lbm.AA):
                out.append((prec, k, layout))
        out.append((prec, lbm.KERNEL_TMA, lbm.PULL2))
    return out


def _channel(prec, kernel, layout, wall, les):
    ch = lbm.Channel.from_case(CASE, precision=prec, wall=wall, layout=layout)
    ch.set_kernel(kernel)
    if les:
        ch.set_les(lbm.COLLISION_MRT, CASE.u_tau, 26.0)
    ch.init_channel(workload.u_mean_profile(CASE), workload.noise_amplitude(CASE), CASE.seed)
    return ch


@pytest.mark.parametrize("les", [False, True])
@pytest.mark.parametrize("wall", [workload.WALL_BB, workload.WALL_WFB])
@pytest.mark.parametrize("prec,kernel,layout", _forms())
def test_back_to_back_equals_separated(prec, kernel, layout, wall, les):
    a = _channel(prec, kernel, layout, wall, les)
    b = _channel(prec, kernel, layout, wall, les)
    t = 0
    for n in RUNS:
        a.step(n)
        for _ in range(n):
            b.step(1)
            b.populations()          # host copy between the steps: no overlap
        t += n
        fa, fb = a.populations(), b.populations()
        assert np.array_equal(fa, fb), (t, prec, kernel, layout, wall, les)
        assert np.array_equal(a.wall_stress(), b.wall_stress()), (t, "tau_w")
    a.close()
    b.close()
