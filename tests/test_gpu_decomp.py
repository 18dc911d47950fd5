"""The z decomposition on the GPU library: every slab of a 2- and 3-way split
held as its own context in one process (the in-process transport; host or
device halo buffers), against the single-domain context of the same form --
bit for bit on the exact FP64 form, to roundoff on the contracted ones --
with identical CFL time steps.  A split over several GPUs runs the same
driver with torch.distributed (NCCL) between processes; its exchange and
reduction are exercised on the CPU with gloo (tests/test_decomp.py)."""
import numpy as np
import pytest

from gpu_util import make_gpu, rel_l1
from paper_1607_02214_gb300 import decomp, inputs, ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


class DeviceTransport(decomp.LocalTransport):
    """In-process halos in device memory."""

    def empty(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
@pytest.mark.parametrize("world,transport", [(2, decomp.LocalTransport), (3, DeviceTransport)])
def test_split_magnetosphere_matches_the_single_domain(precision, world, transport):
    pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    ref = make_gpu(pr, precision)

    def engine(lp):
        c = ppmlr.Context.from_problem(lp, precision)
        c.set_state(lp.U0)
        return c
    run = decomp.ZSlabRun(pr, world, list(range(world)), engine, transport())
    for k in range(6):
        dt = run.cfl_dt(pr.cfl)
        assert dt == ref.cfl_dt(pr.cfl), k
        run.step(dt)
        ref.step(dt)
    for e in run.engines:
        e.check()
    U = np.concatenate([run.owned_state(i) for i in range(world)], axis=1)
    if precision == ppmlr.PPMLR_FP64_EXACT:
        assert np.array_equal(U, ref.get_state())
    else:
        assert np.max(rel_l1(U, ref.get_state())) <= (1e-12 if precision == ppmlr.PPMLR_FP64 else 1e-6)


def test_layer_copies_bounds_and_round_trip():
    import torch
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    c = make_gpu(pr)
    L = c.get_layers(5, 7)
    assert np.array_equal(L, pr.U0[:, 5:12])
    dev = torch.from_numpy(np.ascontiguousarray(pr.U0[:, 20:27] * 2.0)).cuda()
    c.set_layers(20, dev)
    out = torch.empty_like(dev)
    c.get_layers(20, 7, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, dev)
    assert np.array_equal(c.get_state()[:, :20], pr.U0[:, :20])
    for k0, nk in ((-1, 2), (29, 2), (0, 31)):
        with pytest.raises(ppmlr.PPMLRError):
            c.get_layers(k0, nk)
