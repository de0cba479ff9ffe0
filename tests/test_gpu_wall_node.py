"""The full-way (wall-node) WFB on the GPU against the oracle: the one-, two-
and four-cell kernels (the four-cell step runs its node rows with the two-cell
wall tile), FP32 and FP16 storage, BGK and MRT, ragged grids down to one fluid
layer, the batch, and the kernel form and layout that have no wall-node form."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import check_state, floors, reference

pytestmark = pytest.mark.gpu

# the parity configuration (tau0 0.52, C_s 0.1) on wall nodes: 64 x 33 x 32,
# D = 16 between the wall nodes as in the 64 x 32 x 32 halfway case
NODE_C1 = workload.CASES["c1"].with_(name="c1 on wall nodes 64x33x32", ny=33, wall=workload.WALL_WFB_NODE)
# first fluid node at y+ = 40 (the log region of the wall laws), tau0 = 0.50014
NODE = workload.derive_channel("wall-node channel 64x33x32", 64, 33, 32, 640.0,
                               wall=workload.WALL_WFB_NODE, seed=23)
RAGGED = [NODE.with_(nx=37, ny=6, nz=5), NODE.with_(nx=2, ny=3, nz=3), NODE.with_(nx=34, ny=4, nz=3),
          NODE.with_(nx=130, ny=5, nz=2)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def _channel(case, precision, kernel):
    ch = lbm.Channel.from_case(case, precision=precision)
    ch.set_kernel(kernel)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    return ch


FORMS = [(lbm.FP32, lbm.KERNEL_PAIR), (lbm.FP32, lbm.KERNEL_CELL), (lbm.FP16_SHIFTED, lbm.KERNEL_PAIR),
         (lbm.FP16_SHIFTED, lbm.KERNEL_CELL), (lbm.FP16_SHIFTED, lbm.KERNEL_QUAD)]


@pytest.mark.parametrize("precision,kernel", FORMS)
def test_wall_node_parity_100_steps(precision, kernel):
    ref = reference(NODE_C1, (100,))[100]
    fl = floors(NODE_C1, (100,), precision)[100]
    ch = _channel(NODE_C1, precision, kernel)
    assert ch.kernel == kernel
    ch.step(100)
    check_state(ch, ref, fl, precision, NODE_C1.wall, populations=True, tag=kernel)
    ch.close()


@pytest.mark.parametrize("precision,kernel", FORMS)
def test_wall_node_mrt_parity_100_steps(precision, kernel):
    """The paper's LES operator (MRT, Smagorinsky, van Driest damping with the
    distance to the nearer wall node) with the full-way WFB, against the
    oracle."""
    les = (lbm.COLLISION_MRT, NODE_C1.u_tau, 26.0)
    ref = reference(NODE_C1, (100,), None, les)[100]
    fl = floors(NODE_C1, (100,), precision, None, les)[100]
    ch = lbm.Channel.from_case(NODE_C1, precision=precision)
    ch.set_kernel(kernel)
    ch.set_les(*les)
    ch.init_channel(workload.u_mean_profile(NODE_C1), workload.noise_amplitude(NODE_C1), NODE_C1.seed)
    ch.step(100)
    check_state(ch, ref, fl, precision, NODE_C1.wall, populations=True, tag=("mrt", kernel))
    ch.close()


@pytest.mark.parametrize("precision,kernel", FORMS)
def test_wall_node_log_region_100_steps(precision, kernel):
    """Wall law in its log region (R ~ 500) at tau0 near 1/2, where the
    storage rounding of a weakly damped FP16 run accumulates: every quantity
    against its measured storage-rounding floor."""
    ref = reference(NODE, (100,))[100]
    fl = floors(NODE, (100,), precision)[100]
    ch = _channel(NODE, precision, kernel)
    ch.step(100)
    check_state(ch, ref, fl, precision, NODE.wall, populations=True, tag=kernel)
    ch.close()


@pytest.mark.parametrize("case", RAGGED, ids=lambda c: f"{c.nx}x{c.ny}x{c.nz}")
def test_wall_node_ragged(case):
    ref = reference(case, (40,))[40]
    fl = floors(case, (40,), lbm.FP32)[40]
    for kernel in ([lbm.KERNEL_PAIR, lbm.KERNEL_CELL] if case.nx % 2 == 0 else [lbm.KERNEL_CELL]):
        ch = _channel(case, lbm.FP32, kernel)
        ch.step(40)
        check_state(ch, ref, fl, lbm.FP32, case.wall, populations=True, tag=kernel)
        ch.close()


def test_wall_node_log_law_and_mass():
    case = NODE.with_(wall_law=lbm.LAW_LOG)
    ref = reference(case, (60,))[60]
    fl = floors(case, (60,), lbm.FP32)[60]
    ch = _channel(case, lbm.FP32, lbm.KERNEL_PAIR)
    m0 = ch.conservation()[0]
    ch.step(60)
    check_state(ch, ref, fl, lbm.FP32, case.wall, populations=True)
    assert abs(ch.conservation()[0] - m0) <= 1e-6 * m0
    ch.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_wall_node_batch_member_equals_channel(precision):
    members = [NODE.with_(seed=41), NODE.with_(nx=66, ny=9, nz=4, seed=42, wall=workload.WALL_WFB)]
    b = lbm.Batch(members, precision=precision)
    for m, c in zip(b.members, members):
        m.init_channel(workload.u_mean_profile(c), workload.noise_amplitude(c), c.seed)
    b.step(25)
    for i, c in enumerate(members):
        ch = _channel(c, precision, lbm.KERNEL_PAIR)
        ch.step(25)
        assert np.array_equal(b.members[i].populations(), ch.populations()), i
        assert np.array_equal(b.members[i].wall_stress(), ch.wall_stress()), i
        ch.close()
    b.close()


@pytest.mark.parametrize("precision", [lbm.FP16_SHIFTED, lbm.FP32])
def test_wall_node_mrt_forms_agree(precision):
    """MRT + van Driest on wall nodes: every kernel form the grid allows gives
    the same bits (the four-cell step with the two-cell node rows included)."""
    forms = [lbm.KERNEL_PAIR] + ([lbm.KERNEL_QUAD] if precision == lbm.FP16_SHIFTED else [])
    out = []
    for k in forms:
        ch = lbm.Channel.from_case(NODE, precision=precision)
        ch.set_kernel(k)
        ch.set_les(lbm.COLLISION_MRT, NODE.u_tau, 26.0)
        ch.init_channel(workload.u_mean_profile(NODE), workload.noise_amplitude(NODE), NODE.seed)
        ch.step(37)
        out.append((ch.populations(), ch.wall_stress()))
        ch.close()
    for f, tw in out[1:]:
        assert np.array_equal(f, out[0][0]) and np.array_equal(tw, out[0][1])


def test_wall_node_rejects_other_forms():
    ch = lbm.Channel.from_case(NODE, precision=lbm.FP16_SHIFTED)
    assert ch.kernel == lbm.KERNEL_QUAD          # AUTO picks the four-cell form
    with pytest.raises(lbm.LbmError):
        ch.set_kernel(lbm.KERNEL_TMA)
    ch.close()
    with pytest.raises(lbm.LbmError):
        lbm.Channel.from_case(NODE, layout=lbm.AA)
    with pytest.raises(lbm.LbmError):
        lbm.Channel.from_case(NODE.with_(ny=2))
