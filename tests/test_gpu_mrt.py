"""MRT collision and van Driest damping on the GPU against the oracle (the
paper's LES operator of Sec. 3.1: MRT, standard Smagorinsky, van Driest)."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import check_state, floors, reference

pytestmark = pytest.mark.gpu

SMALL = workload.CASES["c1"]
A_PLUS = 26.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("damping", [False, True])
@pytest.mark.parametrize("kernel", [lbm.KERNEL_PAIR, lbm.KERNEL_CELL, lbm.KERNEL_QUAD, lbm.KERNEL_TMA])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("wall", [workload.WALL_WFB, workload.WALL_BB])
def test_mrt_parity_100_steps(wall, precision, kernel, damping):
    if kernel == lbm.KERNEL_QUAD and precision != lbm.FP16_SHIFTED:
        pytest.skip("the four-cell kernel serves FP16 storage only")
    case = SMALL
    les = (lbm.COLLISION_MRT, case.u_tau if damping else 0.0, A_PLUS if damping else 0.0)
    ref = reference(case, (100,), wall, les)[100]
    fl = floors(case, (100,), precision, wall, les)[100]
    ch = lbm.Channel.from_case(case, precision=precision, wall=wall)
    ch.set_kernel(kernel)
    ch.set_les(*les)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    ch.step(100)
    check_state(ch, ref, fl, precision, wall, populations=True, tag=kernel)
    ch.close()


def test_mrt_differs_from_bgk_and_damping_matters():
    """Guards against a silently ignored operator switch."""
    case = SMALL
    res = {}
    for name, coll, damp in (("bgk", lbm.COLLISION_BGK, False), ("mrt", lbm.COLLISION_MRT, False),
                             ("mrt_vd", lbm.COLLISION_MRT, True)):
        ch = lbm.Channel.from_case(case)
        ch.set_les(coll, case.u_tau if damp else 0.0, A_PLUS if damp else 0.0)
        ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
        ch.step(30)
        res[name] = ch.moments()[1]
        ch.close()
    assert rel(res["mrt"], res["bgk"]) > 1e-6
    assert rel(res["mrt_vd"], res["mrt"]) > 1e-7


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_batch_mrt_members_equal_single_channels(precision):
    cases = [SMALL.with_(nx=64, ny=8, nz=6, seed=21), SMALL.with_(nx=96, ny=12, nz=4, seed=22, tau=0.55)]
    b = lbm.Batch(cases, precision=precision)
    b.set_les(lbm.COLLISION_MRT, [c.u_tau for c in cases], A_PLUS)
    for m, c in zip(b.members, cases):
        m.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
    b.step(25)
    for i, c in enumerate(cases):
        ch = lbm.Channel.from_case(c, precision=precision)
        ch.set_kernel(lbm.KERNEL_PAIR)
        ch.set_les(lbm.COLLISION_MRT, c.u_tau, A_PLUS)
        ch.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
        ch.step(25)
        assert np.array_equal(b.members[i].populations(), ch.populations()), i
        ch.close()
    b.close()


def test_set_les_rejects_bad_arguments():
    ch = lbm.Channel.from_case(SMALL.with_(nx=8, ny=4, nz=2))
    for args in ((7, 0.0, 0.0), (lbm.COLLISION_MRT, 1e-3, 0.0), (lbm.COLLISION_MRT, 0.0, 26.0),
                 (lbm.COLLISION_BGK, -1.0, 26.0)):
        with pytest.raises(lbm.LbmError):
            ch.set_les(*args)
    ch.close()
