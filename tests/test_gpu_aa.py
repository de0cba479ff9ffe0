"""The single-lattice AA layout against the two-lattice pull layout and the
oracle.

Both layouts apply the same arithmetic to the same values in the same order
(only where the values live differs), so populations, moments, wall stress,
statistics and conservation sums must agree bitwise after any number of
steps: even counts (natural phase), odd counts (the state sits in the
opposite slots of the pull sources), across CUDA-graph chunks started from
either phase, on ragged grids and for every wall kind."""
import numpy as np
import pytest

import oracle
from paper_2009_04352_gb300 import lbm, workload
from parity import check_state, floors, reference

pytestmark = pytest.mark.gpu

SMALL = workload.CASES["c1"]
WALLS = [workload.WALL_BB, workload.WALL_WFB, workload.WALL_FREESLIP]
# ragged rows, rows shorter than a warp, one pair or one quad per row, ny = 2
RAGGED = [SMALL.with_(nx=37, ny=6, nz=5), SMALL.with_(nx=2, ny=6, nz=3), SMALL.with_(nx=4, ny=5, nz=2),
          SMALL.with_(nx=34, ny=2, nz=3), SMALL.with_(nx=66, ny=4, nz=3), SMALL.with_(nx=300, ny=3, nz=2),
          SMALL.with_(nx=1, ny=8, nz=1), SMALL.with_(nx=132, ny=5, nz=2)]
CHECKPOINTS = (1, 2, 3, 20, 37)   # 17 steps from phase 1 run a graph chunk started there


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()
    oracle.build()


def _kernels(case, precision):
    ks = [lbm.KERNEL_CELL]
    if case.nx % 2 == 0:
        ks.append(lbm.KERNEL_PAIR)
    if case.nx % 4 == 0 and precision == lbm.FP16_SHIFTED:
        ks.append(lbm.KERNEL_QUAD)
    return ks


def _channel(case, wall, precision, layout, kernel):
    ch = lbm.Channel.from_case(case, precision=precision, wall=wall, layout=layout)
    ch.set_kernel(kernel)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    return ch


def _snapshots(ch, checkpoints):
    out, t = [], 0
    for c in checkpoints:
        ch.step(c - t)
        t = c
        rho, u = ch.moments()
        out.append(dict(f=ch.populations(), rho=rho, u=u, tw=ch.wall_stress(), cons=ch.conservation()))
    return out


def _assert_same(a, b, what):
    for i, (x, y) in enumerate(zip(a, b)):
        for k in x:
            assert np.array_equal(x[k], y[k]), (what, CHECKPOINTS[i], k)


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("wall", WALLS)
def test_aa_equals_pull_bitwise(wall, precision):
    case = SMALL
    for kernel in _kernels(case, precision):
        pull = _channel(case, wall, precision, lbm.PULL2, kernel)
        aa = _channel(case, wall, precision, lbm.AA, kernel)
        assert aa.kernel == kernel
        _assert_same(_snapshots(pull, CHECKPOINTS), _snapshots(aa, CHECKPOINTS), kernel)
        pull.close()
        aa.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("case", RAGGED, ids=lambda c: f"{c.nx}x{c.ny}x{c.nz}")
@pytest.mark.parametrize("wall", WALLS)
def test_aa_equals_pull_ragged(case, wall, precision):
    for kernel in _kernels(case, precision):
        pull = _channel(case, wall, precision, lbm.PULL2, kernel)
        aa = _channel(case, wall, precision, lbm.AA, kernel)
        _assert_same(_snapshots(pull, CHECKPOINTS), _snapshots(aa, CHECKPOINTS), (case.nx, kernel))
        pull.close()
        aa.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_aa_parity_with_oracle_100_steps(precision):
    case = SMALL
    checkpoints = (98, 99)             # both phases; an odd count leaves the AA state in phase 1
    ref = reference(case, checkpoints, workload.WALL_WFB)
    fl = floors(case, checkpoints, precision, workload.WALL_WFB)
    ch = lbm.Channel.from_case(case, precision=precision, layout=lbm.AA)
    ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
    t = 0
    for c in checkpoints:
        ch.step(c - t)
        t = c
        check_state(ch, ref[c], fl[c], precision, workload.WALL_WFB, populations=True, tag=c)
    ch.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
def test_aa_statistics_and_mrt_match_pull(precision):
    """Sampled plane statistics (fused into steps of both kinds) and the MRT +
    van Driest operator."""
    case = SMALL
    res = []
    for layout in (lbm.PULL2, lbm.AA):
        ch = lbm.Channel.from_case(case, precision=precision, layout=layout)
        ch.set_les(lbm.COLLISION_MRT, case.u_tau, 26.0)
        ch.init_channel(workload.u_mean_profile(case), workload.noise_amplitude(case), case.seed)
        ch.set_stats_every(3)
        ch.step(41)
        s, w, n = ch.plane_stats()
        res.append((ch.populations(), s, w, n))
        ch.close()
    (fa, sa, wa, na), (fb, sb, wb, nb) = res
    assert na == nb == 14
    assert np.array_equal(fa, fb)
    if precision == lbm.FP32:
        assert np.array_equal(sa, sb)
    else:
        # the two-lattice FP16 MRT step runs its wall rows in a second launch
        # with the two-cell tile, whose threads and warps add the same cell
        # values (bitwise equal, as the populations show) in another order
        # than the single AA launch; the warp sums are FP32, so the plane sums
        # agree to a few FP32 roundings of the warp sums
        scale = np.max(np.abs(sa), axis=0)
        assert np.all(np.abs(sa - sb) <= 1e-6 * scale), np.max(np.abs(sa - sb) / scale)
    # tau_w is FP32 arithmetic that the compiler may contract into FMAs
    # differently in two kernel instantiations; under FP16 storage the last-bit
    # difference does not reach the stored populations, only the wall sums,
    # which the FP16 step also adds in another order (see above)
    scale = np.max(np.abs(wa), axis=0)
    assert np.all(np.abs(wa - wb) <= 1e-6 * scale), np.max(np.abs(wa - wb) / scale)


def test_aa_set_populations_at_odd_phase():
    """Populations read at an odd step count and written back restart the run
    in the natural phase; the continuation matches the pull layout's."""
    case = SMALL.with_(nx=66, ny=8, nz=6)
    pull = _channel(case, workload.WALL_WFB, lbm.FP32, lbm.PULL2, lbm.KERNEL_PAIR)
    aa = _channel(case, workload.WALL_WFB, lbm.FP32, lbm.AA, lbm.KERNEL_PAIR)
    pull.step(5)
    aa.step(5)
    f = aa.populations()
    assert np.array_equal(f, pull.populations())
    aa.set_populations(f)
    pull.set_populations(f)
    assert np.array_equal(aa.populations(), f)
    pull.step(7)
    aa.step(7)
    assert np.array_equal(aa.populations(), pull.populations())
    pull.close()
    aa.close()


def test_aa_noalloc_profile_matches_pull():
    import torch
    case = SMALL
    outs = []
    for layout in (lbm.PULL2, lbm.AA):
        ch = _channel(case, workload.WALL_WFB, lbm.FP32, layout, lbm.KERNEL_PAIR)
        ch.step(7)
        out = torch.zeros((case.ny, lbm.K_STATS), dtype=torch.float64, device="cuda")
        lbm.lbm_plane_profile_noalloc(ch.handle, out.data_ptr())
        ch.sync()
        outs.append(out.cpu().numpy())
        ch.close()
    assert np.array_equal(outs[0], outs[1])


def test_aa_rejects_pipelined_kernel_and_halves_memory():
    import torch
    case = workload.CASES["c2"]
    aa = lbm.Channel.from_case(case, layout=lbm.AA)
    with pytest.raises(lbm.LbmError):
        aa.set_kernel(lbm.KERNEL_TMA)
    aa.close()
    used = {}
    for layout in (lbm.PULL2, lbm.AA):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ch = lbm.Channel.from_case(case, layout=layout)
        ch.sync()
        used[layout] = free0 - torch.cuda.mem_get_info()[0]
        ch.close()
    lattice = 19 * case.cells * 4
    assert used[lbm.PULL2] >= 2 * lattice
    assert used[lbm.AA] < 1.25 * lattice


@pytest.mark.parametrize("case", [SMALL, SMALL.with_(nx=132, ny=5, nz=2), SMALL.with_(nx=4, ny=5, nz=2)],
                         ids=lambda c: f"{c.nx}x{c.ny}x{c.nz}")
def test_aa_kernel_switch_mid_run(case):
    """Switching the kernel form of an FP16 AA channel in the middle of a run,
    at either phase, keeps the state: each stretch equals the two-lattice
    channel run with the same forms."""
    pull = _channel(case, workload.WALL_WFB, lbm.FP16_SHIFTED, lbm.PULL2, lbm.KERNEL_QUAD)
    aa = _channel(case, workload.WALL_WFB, lbm.FP16_SHIFTED, lbm.AA, lbm.KERNEL_QUAD)
    t = 0
    for kernel, n in ((lbm.KERNEL_QUAD, 7), (lbm.KERNEL_PAIR, 5), (lbm.KERNEL_CELL, 4), (lbm.KERNEL_QUAD, 6)):
        aa.set_kernel(kernel)
        pull.set_kernel(kernel)
        aa.step(n)
        pull.step(n)
        t += n
        assert np.array_equal(aa.populations(), pull.populations()), (kernel, t)
        assert np.array_equal(aa.wall_stress(), pull.wall_stress()), (kernel, t)
        assert np.array_equal(aa.moments()[1], pull.moments()[1]), (kernel, t)
    aa.close()
    pull.close()
