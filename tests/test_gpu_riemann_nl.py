"""The nonlinear (two-shock, fast-mode) Riemann solver on the GPU against the
oracle's: bit for bit on the exact FP64 path, to the FP64 and mixed
tolerances on the other paths, on a strong colliding flow, Brio-Wu and the
magnetosphere; the option is honoured by graph-replayed runs and rejected
outside its range."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle, rel_l1
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

ITERS = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def colliding_flow():
    return inputs.shock_tube_1d(200, (1.0, 3.0, 0, 0, 0.5, 0.8, 0, 1.0), (1.0, -3.0, 0, 0, 0.5, -0.4, 0, 1.0),
                                5.0 / 3.0)


CASES = {
    "colliding_flow": colliding_flow,
    "brio_wu": lambda: inputs.brio_wu_3d((32, 32, 32)),
    "magnetosphere": lambda: inputs.magnetosphere(n=(48, 40, 36), h0=1.0),
}


def pair(pr, precision, nsteps):
    o = make_oracle(pr)
    o.set_riemann(ITERS)
    g = make_gpu(pr, precision)
    g.set_riemann_solver(ITERS)
    for _ in range(nsteps):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    return o, g


@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_path_is_bit_identical_to_the_oracle(case):
    o, g = pair(CASES[case](), ppmlr.PPMLR_FP64_EXACT, 6)
    assert np.array_equal(g.get_state(), o.get_state())


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_path_within_tolerance(case):
    o, g = pair(CASES[case](), ppmlr.PPMLR_FP64, 10)
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= 1e-11, err


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_path_within_tolerance(case):
    o, g = pair(CASES[case](), ppmlr.PPMLR_MIXED, 10)
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= 1e-5, err


def test_option_changes_the_solution_and_zero_is_the_default():
    pr = colliding_flow()
    a, b, c = make_gpu(pr), make_gpu(pr), make_gpu(pr)
    b.set_riemann_solver(0)
    c.set_riemann_solver(ITERS)
    for _ in range(5):
        dt = a.cfl_dt(pr.cfl)
        for g in (a, b, c):
            g.step(dt)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.max(rel_l1(c.get_state(), a.get_state())) > 1e-6
    for bad in (-1, 17):
        with pytest.raises(ppmlr.PPMLRError):
            a.set_riemann_solver(bad)


def test_graph_run_uses_the_nonlinear_solver():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    a, b = make_gpu(pr), make_gpu(pr)
    a.run(pr.cfl, 4, graph_steps=2)                  # graphs captured with the two-wave solver
    b.step_cfl(pr.cfl, 4)
    for g in (a, b):
        g.set_riemann_solver(ITERS)                  # drops the captured graphs
    a.run(pr.cfl, 4, graph_steps=2)
    b.step_cfl(pr.cfl, 4)
    assert np.array_equal(a.get_state(), b.get_state())


def test_ensemble_instances_use_the_nonlinear_solver():
    from test_gpu_ensemble import small_ensemble
    probs = small_ensemble(3)[:3]
    ens = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_FP64_EXACT)
    ens.set_riemann_solver(ITERS)
    for i, p in enumerate(probs):
        ens.set_state(i, p.U0)
    ens.step(0.4, 3)                                 # graph replay, per-instance device dt
    for i, p in enumerate(probs):
        o = make_oracle(p)
        o.set_riemann(ITERS)
        for _ in range(3):
            assert o.step(o.cfl_dt(0.4)) == 0
        assert np.array_equal(ens.get_state(i), o.get_state()), i
    with pytest.raises(ppmlr.PPMLRError):
        ens.set_riemann_solver(17)
