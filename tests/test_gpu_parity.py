"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Relative L_inf (max |gpu - oracle| / max |oracle| over cells and components)
of the velocity u, the density deviation rho - 1, the population deviations
f - w and the wall stress, bounded by the benchmark's tolerance (1e-5 FP32, 5e-3
FP16 storage) or by twice the measured storage-rounding floor, whichever is
larger (tests/parity.py states the bounds and how the floor is measured)."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import W, check_state, floors, reference, rel

pytestmark = pytest.mark.gpu

WALLS = [workload.WALL_BB, workload.WALL_WFB, workload.WALL_FREESLIP]
rel_linf = rel


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def oracle_run(case, wall, checkpoints, stats_every=0):
    """Moments, wall stress and populations of the oracle at each checkpoint."""
    return reference(case, checkpoints, wall, stats_every=stats_every)


def gpu_channel(case, wall, precision, kernel=lbm.KERNEL_AUTO):
    ch = lbm.Channel.from_case(case, precision=precision, wall=wall)
    if kernel != lbm.KERNEL_AUTO:
        ch.set_kernel(kernel)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    return ch


SMALL = workload.CASES["c1"]                       # 64 x 32 x 32, tau0 0.52
# odd nx runs the one-cell kernel, even nx the two-cell kernel; rows shorter
# than a warp, rows ending inside a warp, a single column, ny = 2 (both layers
# are wall layers)
RAGGED = [SMALL.with_(nx=37, ny=6, nz=5), SMALL.with_(nx=1, ny=8, nz=1),
          SMALL.with_(nx=33, ny=2, nz=3), SMALL.with_(nx=130, ny=5, nz=2),
          SMALL.with_(nx=2, ny=6, nz=3), SMALL.with_(nx=66, ny=4, nz=3),
          SMALL.with_(nx=34, ny=2, nz=3), SMALL.with_(nx=300, ny=3, nz=2),
          SMALL.with_(nx=64, ny=2, nz=3), SMALL.with_(nx=192, ny=5, nz=2),
          SMALL.with_(nx=128, ny=3, nz=1)]
KERNELS = [lbm.KERNEL_TMA, lbm.KERNEL_PAIR, lbm.KERNEL_CELL, lbm.KERNEL_QUAD]


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_init_matches_oracle(precision):
    case = SMALL
    ref = oracle_run(case, workload.WALL_WFB, (0,))[0]
    ch = gpu_channel(case, workload.WALL_WFB, precision)
    f = ch.populations()
    dev_ref = ref["f"] - W
    # one rounding of the deviation to the storage precision
    ulp = 2.0 ** -24 if precision == lbm.FP32 else 2.0 ** -11
    assert np.max(np.abs((f - W) - dev_ref)) <= ulp * np.max(np.abs(dev_ref)) + 1e-12
    ch.close()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("wall", WALLS)
def test_parity_100_steps(wall, precision, kernel):
    """64x32x32 channel, tau0 0.52, C_s 0.1, seeded log-law + 10% noise: 100 steps."""
    if kernel == lbm.KERNEL_QUAD and precision != lbm.FP16_SHIFTED:
        pytest.skip("the four-cell kernel serves FP16 storage only")
    case = SMALL
    checkpoints = (1, 10, 50, 100)
    ref = oracle_run(case, wall, checkpoints)
    fl = floors(case, checkpoints, precision, wall)
    ch = gpu_channel(case, wall, precision, kernel)
    assert ch.kernel == kernel
    t = 0
    for c in checkpoints:
        ch.step(c - t)
        t = c
        check_state(ch, ref[c], fl[c], precision, wall, populations=(c == 100), tag=(c, kernel))
    ch.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("case", RAGGED, ids=lambda c: f"{c.nx}x{c.ny}x{c.nz}")
@pytest.mark.parametrize("wall", WALLS)
def test_parity_ragged(case, wall, precision):
    checkpoints = (1, 7, 20)
    ref = oracle_run(case, wall, checkpoints)
    fl = floors(case, checkpoints, precision, wall)
    ch = gpu_channel(case, wall, precision)
    t = 0
    for c in checkpoints:
        ch.step(c - t)
        t = c
        check_state(ch, ref[c], fl[c], precision, wall, populations=(c == 20), tag=c)
    ch.close()


@pytest.mark.parametrize("wall", [workload.WALL_BB, workload.WALL_WFB])
def test_plane_stats_and_conservation(wall):
    case = SMALL.with_(nx=48, ny=12, nz=10)
    L = oracle.Lattice.from_case(case, stats_every=3, wall=wall)
    L.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    L.step(30)
    st_o, w_o, n_o = L.plane_stats()
    cons_o = L.conservation()

    ch = gpu_channel(case, wall, lbm.FP32)
    ch.set_stats_every(3)
    ch.step(30)
    st_g, w_g, n_g = ch.plane_stats()
    cons_g = ch.conservation()
    assert n_g == n_o == 10
    # columns: rho and u moments compared relative to each column's scale
    for k in range(st_o.shape[1]):
        ref = st_o[:, k]
        if k == 0:
            assert np.max(np.abs(st_g[:, 0] - ref)) <= 1e-6 * np.max(np.abs(ref))
        else:
            assert rel_linf(st_g[:, k], ref) <= 1e-4, k
    assert rel_linf(w_g, w_o) <= 1e-4
    assert abs(cons_g[0] - cons_o[0]) <= 1e-7 * cons_o[0]
    assert np.max(np.abs(cons_g[1:] - cons_o[1:])) <= 1e-5 * np.max(np.abs(cons_o[1:]))
    # reset clears the accumulators
    ch.plane_stats(reset=True)
    st2, w2, n2 = ch.plane_stats()
    assert n2 == 0 and np.all(st2 == 0.0) and np.all(w2 == 0.0)
    ch.close()


def test_graph_replay_matches_single_launches():
    """Chunked CUDA-graph replay gives bit-identical results to one launch per step."""
    case = SMALL.with_(nx=40, ny=10, nz=6)
    a = gpu_channel(case, workload.WALL_WFB, lbm.FP32)
    b = gpu_channel(case, workload.WALL_WFB, lbm.FP32)
    a.step(70)
    for _ in range(70):
        b.step(1)
    assert a.step_count == b.step_count == 70
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.wall_stress(), b.wall_stress())
    a.close()
    b.close()


@pytest.mark.parametrize("wall", WALLS)
def test_gpu_momentum_budget(wall):
    """Per step the x and z momentum change by N F + sum of the wall stresses
    (Eq. 9 / 12b summed), checked on the GPU alone in FP64 reductions."""
    case = SMALL.with_(nx=32, ny=8, nz=16, force=(2e-6, 0.0, -1e-6))
    ch = gpu_channel(case, wall, lbm.FP32)
    p0 = ch.conservation()
    for _ in range(5):
        ch.step(1)
        p1 = ch.conservation()
        tw = ch.wall_stress().astype(np.float64)
        for c, comp in ((1, 0), (3, 1)):
            expect = case.cells * case.force[c - 1] + tw[..., comp].sum()
            assert abs((p1[c] - p0[c]) - expect) <= 1e-3 * max(abs(expect), case.cells * 1e-6), (wall, c)
        assert abs(p1[0] - p0[0]) <= 1e-9 * p0[0]
        p0 = p1
    ch.close()


def test_moments_on_device():
    import torch
    case = SMALL.with_(nx=20, ny=6, nz=4)
    ch = gpu_channel(case, workload.WALL_WFB, lbm.FP32)
    ch.step(3)
    rho_h, u_h = ch.moments()
    rho_d, u_d = ch.moments(device=True)
    torch.cuda.synchronize()
    assert np.array_equal(rho_d.cpu().numpy(), rho_h)
    assert np.array_equal(u_d.cpu().numpy(), u_h)
    ch.close()


def test_set_populations_round_trip():
    case = SMALL.with_(nx=24, ny=7, nz=5)
    ref = oracle_run(case, workload.WALL_WFB, (3,))[3]
    ch = lbm.Channel.from_case(case)
    ch.set_populations(ref["f"])
    f = ch.populations()
    dev = ref["f"] - W
    assert np.max(np.abs(f - ref["f"])) <= 2.0 ** -24 * np.max(np.abs(dev)) + 1e-15
    ch.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_full_size_bench_grid(precision):
    """256x64x128 (the benchmark's FP32 channel), launch configuration as benched:
    three steps compared with the oracle on every cell."""
    case = workload.CASES["c2"]
    ref = oracle_run(case, workload.WALL_WFB, (3,))[3]
    fl = floors(case, (3,), precision, workload.WALL_WFB)[3]
    ch = gpu_channel(case, workload.WALL_WFB, precision)
    ch.step(3)
    check_state(ch, ref, fl, precision, workload.WALL_WFB, populations=True)
    ch.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_pipelined_and_pair_kernels_agree_bitwise(precision):
    """The warp-pipelined and the two-cell kernels share the collision code and
    must give identical bits; statistics included."""
    case = SMALL.with_(nx=128, ny=8, nz=6)
    a = gpu_channel(case, workload.WALL_WFB, precision, lbm.KERNEL_TMA)
    b = gpu_channel(case, workload.WALL_WFB, precision, lbm.KERNEL_PAIR)
    for ch in (a, b):
        ch.set_stats_every(4)
        ch.step(37)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.wall_stress(), b.wall_stress())
    sa, wa, na = a.plane_stats()
    sb, wb, nb = b.plane_stats()
    assert na == nb == 10
    assert np.allclose(sa, sb, rtol=1e-12, atol=1e-15) and np.allclose(wa, wb, rtol=1e-12, atol=1e-18)
    a.close()
    b.close()


def test_kernel_selection_rules():
    case = SMALL.with_(nx=66, ny=4, nz=2)
    ch = lbm.Channel.from_case(case)
    assert ch.kernel == lbm.KERNEL_PAIR
    with pytest.raises(lbm.LbmError):
        ch.set_kernel(lbm.KERNEL_TMA)
    ch.close()
    ch = lbm.Channel.from_case(case.with_(nx=37))
    assert ch.kernel == lbm.KERNEL_CELL
    with pytest.raises(lbm.LbmError):
        ch.set_kernel(lbm.KERNEL_PAIR)
    ch.close()
    ch = lbm.Channel.from_case(case.with_(nx=128))
    assert ch.kernel == lbm.KERNEL_PAIR
    ch.set_kernel(lbm.KERNEL_TMA)
    assert ch.kernel == lbm.KERNEL_TMA
    with pytest.raises(lbm.LbmError):
        ch.set_kernel(lbm.KERNEL_QUAD)          # FP32 storage
    ch.close()
    ch = lbm.Channel.from_case(case.with_(nx=128), precision=lbm.FP16_SHIFTED)
    assert ch.kernel == lbm.KERNEL_QUAD
    ch.close()


def test_quad_and_pair_kernels_agree_bitwise():
    """FP16 four-cell and two-cell kernels run the same per-cell arithmetic."""
    case = SMALL.with_(nx=300, ny=8, nz=6)
    a = gpu_channel(case, workload.WALL_WFB, lbm.FP16_SHIFTED, lbm.KERNEL_QUAD)
    b = gpu_channel(case, workload.WALL_WFB, lbm.FP16_SHIFTED, lbm.KERNEL_PAIR)
    for ch in (a, b):
        ch.set_stats_every(4)
        ch.step(37)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.wall_stress(), b.wall_stress())
    sa, wa, na = a.plane_stats()
    sb, wb, nb = b.plane_stats()
    assert na == nb == 10
    # the plane sums add the same cell values per thread and warp in FP32 in
    # another grouping (four against two cells per thread), and the FP32 wall
    # stress of a sampled step may differ in its last bit between the two forms
    # (FP16 storage of the populations hides it): they agree to a few FP32
    # roundings of the warp sums
    for got, ref in ((sa, sb), (wa, wb)):
        scale = np.max(np.abs(ref), axis=0)
        assert np.all(np.abs(got - ref) <= 1e-6 * scale), np.max(np.abs(got - ref) / scale)
    a.close()
    b.close()
