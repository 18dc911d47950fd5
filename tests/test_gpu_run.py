"""Long runs: graph-replayed steps give the results of direct launches bit for
bit, the simulated time is the sum of the steps' dt, checkpoints resume a run
bit for bit and damaged or mismatched checkpoints are refused with the state
unchanged, and a 200-step run of the exact FP64 path stays bit-identical to
the oracle."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle, rel_l1
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

PRECISIONS = [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def small_magnetosphere():
    return inputs.magnetosphere(n=(40, 34, 30), h0=1.0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_graph_run_equals_direct_steps(precision):
    pr = small_magnetosphere()
    a, b = make_gpu(pr, precision), make_gpu(pr, precision)
    if precision == ppmlr.PPMLR_MIXED:           # TMA-staged y/z sweeps inside the graphs too
        for c in (a, b):
            for axis in (1, 2):
                c.set_tiles(axis, pr.edges[axis].size - 1, 2)
                c.set_sweep_form(axis, 2)
    a.step_cfl(pr.cfl, 1)                        # start the graphs at an odd step
    b.step_cfl(pr.cfl, 1)
    a.run(pr.cfl, 11, graph_steps=4)             # two replays and three direct steps
    b.step_cfl(pr.cfl, 11)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.diagnostics() == b.diagnostics()
    assert a.time == b.time
    a.run(pr.cfl, 8, graph_steps=4)              # cached graphs of the other parity
    b.run(pr.cfl, 8, graph_steps=0)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.time == b.time and a.diagnostics()["step"] == 20


def test_time_is_the_sum_of_the_steps_dt():
    pr = small_magnetosphere()
    g = make_gpu(pr)
    t = 0.0
    for _ in range(5):
        g.step_cfl(pr.cfl, 1)
        t += g.last_dt()
    assert g.time == t
    g.step(1e-3)
    assert g.time == t + 1e-3
    g.time = 2.5
    g.run(pr.cfl, 2, graph_steps=2)
    assert g.time > 2.5


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
def test_checkpoint_resume_is_bitwise(tmp_path, precision):
    pr = small_magnetosphere()
    a = make_gpu(pr, precision)
    a.run(pr.cfl, 7, graph_steps=2)
    path = tmp_path / "run.ck"
    a.checkpoint_save(path)
    info = ppmlr.checkpoint_info(path)
    assert info["step"] == 7 and info["n"] == [40, 34, 30] and info["time"] == a.time
    a.run(pr.cfl, 9, graph_steps=2)
    b = ppmlr.Context.from_problem(pr, precision)     # a fresh context, no state set
    b.checkpoint_load(path)
    assert b.diagnostics()["step"] == 7
    b.run(pr.cfl, 9, graph_steps=2)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.time == b.time


def test_damaged_or_foreign_checkpoint_is_refused(tmp_path):
    pr = small_magnetosphere()
    a = make_gpu(pr)
    a.run(pr.cfl, 2, graph_steps=2)
    path = tmp_path / "a.ck"
    a.checkpoint_save(path)
    data = bytearray(path.read_bytes())
    data[len(data) // 2] ^= 0x04
    bad = tmp_path / "bad.ck"
    bad.write_bytes(bytes(data))
    b = make_gpu(pr)
    before = b.get_state()
    with pytest.raises(ppmlr.PPMLRError):
        b.checkpoint_load(bad)
    assert np.array_equal(b.get_state(), before) and b.diagnostics()["step"] == 0
    other = make_gpu(inputs.magnetosphere(n=(40, 34, 32), h0=1.0))
    with pytest.raises(ppmlr.PPMLRError):
        other.checkpoint_load(path)
    stretched = make_gpu(inputs.magnetosphere(n=(40, 34, 30), h0=0.9))   # same size, other edges
    with pytest.raises(ppmlr.PPMLRError):
        stretched.checkpoint_load(path)
    pr_gamma = small_magnetosphere()                                       # same grid, other gamma
    pr_gamma.gamma = 1.4
    other_gamma = make_gpu(pr_gamma)
    before = other_gamma.get_state()
    with pytest.raises(ppmlr.PPMLRError):
        other_gamma.checkpoint_load(path)
    assert np.array_equal(other_gamma.get_state(), before)


def test_long_exact_run_is_bit_identical_to_the_oracle():
    pr = inputs.brio_wu_3d((32, 32, 32))
    o = make_oracle(pr)
    for _ in range(200):
        assert o.step(o.cfl_dt(pr.cfl)) == 0
    g = make_gpu(pr, ppmlr.PPMLR_FP64_EXACT)
    g.run(pr.cfl, 200, graph_steps=16)
    assert np.array_equal(g.get_state(), o.get_state())
    f = make_gpu(pr, ppmlr.PPMLR_FP64)
    f.run(pr.cfl, 200, graph_steps=16)
    err = rel_l1(f.get_state(), o.get_state())
    assert np.max(err) <= 1e-10, err
