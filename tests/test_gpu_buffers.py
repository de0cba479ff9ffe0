"""lbm_create_from_buffers: the population arrays come from the caller (here
torch tensors from its caching allocator). The run must be bitwise the run of
a library-allocated channel, and destroying the handle must leave the
caller's memory alone."""
import numpy as np
import pytest

from paper_2009_04352_gb300 import lbm, workload

pytestmark = pytest.mark.gpu

CASE = workload.CASES["c1"].with_(nx=66, ny=10, nz=6)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_04352_gb300 import build
    build.build()


def _init(ch):
    ch.init_channel(workload.u_mean_profile(CASE), workload.noise_amplitude(CASE), CASE.seed)


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16_SHIFTED])
@pytest.mark.parametrize("layout", [lbm.PULL2, lbm.AA])
def test_buffers_run_equals_owned_run(layout, precision):
    import torch
    nbytes = lbm.lbm_population_bytes(CASE.nx, CASE.ny, CASE.nz, precision)
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(1 if layout == lbm.AA else 2)]
    a = lbm.Channel.from_buffers(CASE, bufs, precision=precision, layout=layout)
    b = lbm.Channel.from_case(CASE, precision=precision, layout=layout)
    for ch in (a, b):
        _init(ch)
        ch.set_stats_every(4)
        ch.step(37)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.wall_stress(), b.wall_stress())
    assert np.array_equal(a.plane_stats()[0], b.plane_stats()[0])
    # the state lives in the caller's tensors
    torch.cuda.synchronize()
    before = [t.clone() for t in bufs]
    assert any(int(t.count_nonzero()) > 0 for t in before)
    a.close()
    b.close()
    torch.cuda.synchronize()
    for t, t0 in zip(bufs, before):
        assert torch.equal(t, t0)


def test_buffers_too_small_rejected():
    import torch
    nbytes = lbm.lbm_population_bytes(CASE.nx, CASE.ny, CASE.nz, lbm.FP32)
    small = torch.empty(nbytes - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        lbm.Channel.from_buffers(CASE, [small], layout=lbm.AA)
