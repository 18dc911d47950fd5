"""The marching form of the mixed-precision sweeps (launch form 3: one thread
per pencil walking it cell by cell) against the FP64 oracle, element by
element, and against the tile form of the same precision.  Covers every
axis, ragged lane groups (pencil counts and nx not multiples of 32), chunked
pencils with a ragged last chunk, periodic / outflow / inflow ghosts, the
dipole, Powell sources and inner sphere, the pressure floor count, the
two-shock Riemann solver, the ionosphere shell's per-cell inner states, the
CFL and non-finite flags, graph replay, and the fall-back to the tile form
when contact steepening is on."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle, rel_l1, run_pair
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5
MIX = ppmlr.PPMLR_MIXED


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def periodic_random(n, seed):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    return inputs.Problem("rand", edges, 5.0 / 3.0, inputs.BoundarySpec(powell=1),
                          inputs.random_smooth_state(n, seed, edges=edges))


def marching(pr, chunks=None):
    g = make_gpu(pr, MIX)
    for axis in range(3):
        g.set_sweep_form(axis, 3)
        if chunks:
            g.set_march_chunk(axis, chunks[axis])
    assert g.sweep_forms() == [3, 3, 3]
    return g


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_sweep_against_oracle(axis):
    pr = periodic_random((37, 29, 23), 3)
    o, g = make_oracle(pr), marching(pr)
    dt = o.cfl_dt(0.4)
    assert o.sweep(axis, dt) == 0
    g.sweep(axis, dt)
    g.check()
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= MIXED_TOL, err
    t = make_gpu(pr, MIX)                        # the tile form of the same precision
    t.sweep(axis, dt)
    assert np.max(rel_l1(g.get_state(), t.get_state())) <= 1e-6


@pytest.mark.parametrize("chunks", [None, (10, 8, 7), (37, 15, 23)])
def test_ragged_periodic_steps_against_oracle(chunks):
    pr = periodic_random((37, 29, 23), 5)
    o = make_oracle(pr)
    g = marching(pr, chunks)
    if chunks:
        assert g.tiles() == (list(chunks), [32, 32, 32])
    for _ in range(6):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    g.check()
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= MIXED_TOL, err


def test_magnetosphere_against_oracle_and_floor_count():
    pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    o = make_oracle(pr)
    g = marching(pr, (17, 40, 12))
    t = make_gpu(pr, MIX)
    for _ in range(20):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
        t.step(dt)
    g.check()
    a, b = g.get_state(), o.get_state()
    assert np.all(np.isfinite(a))
    err = rel_l1(a, b)
    assert np.max(err) <= MIXED_TOL, err
    assert g.diagnostics()["floor_hits"] == t.diagnostics()["floor_hits"]


def test_long_pencils_chunked():
    for n, C in (((300, 4, 3), 97), ((5, 280, 3), 64), ((3, 4, 260), 260)):
        pr = periodic_random(n, 9)
        o = make_oracle(pr)
        g = marching(pr, tuple(C if k == max(n) else k for k in n))
        for _ in range(2):
            dt = o.cfl_dt(pr.cfl)
            assert o.step(dt) == 0
            g.step(dt)
        err = rel_l1(g.get_state(), o.get_state())
        assert np.max(err) <= MIXED_TOL, (n, err)


def test_degenerate_axes_of_one_cell():
    pr = periodic_random((33, 1, 5), 12)
    o = make_oracle(pr)
    g = marching(pr)
    for _ in range(3):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    assert np.max(rel_l1(g.get_state(), o.get_state())) <= MIXED_TOL


def test_two_shock_solver():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    o = make_oracle(pr)
    o.set_riemann(4)
    g = marching(pr)
    g.set_riemann_solver(4)
    for _ in range(6):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    assert np.max(rel_l1(g.get_state(), o.get_state())) <= MIXED_TOL


def test_steepening_falls_back_to_the_tile_form():
    pr = periodic_random((30, 20, 18), 14)
    g = marching(pr)
    g.set_steepening(True)
    t = make_gpu(pr, MIX)
    t.set_steepening(True)
    for _ in range(3):
        dt = t.cfl_dt(0.4)
        g.step(dt)
        t.step(dt)
    assert np.array_equal(g.get_state(), t.get_state())


def test_flags_reported():
    pr = inputs.brio_wu_3d((40, 8, 8))
    U = pr.U0.copy()
    U[7, 3, 4, 5] = np.nan
    g = marching(pr)
    g.set_state(U)
    g.step(1e-3)
    assert g.check(raise_on_error=False) == ppmlr.PPMLR_E_NONFINITE
    g = marching(pr)
    dt = g.cfl_dt(0.4)
    g.step(40 * dt)
    assert g.check(raise_on_error=False) in (ppmlr.PPMLR_E_CFL, ppmlr.PPMLR_E_NONFINITE)


def test_graph_replay_equals_direct_steps():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    a = marching(pr)
    b = marching(pr)
    a.run(pr.cfl, 6, graph_steps=2)
    for _ in range(6):
        b.step_cfl(pr.cfl, 1)
    assert np.array_equal(a.get_state(), b.get_state())


def test_ionosphere_inner_states():
    from oracle import ionosphere as I
    from test_gpu_ionosphere import CFG, developed_state, oracle_cfg
    pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    U = developed_state(pr)
    g = marching(pr)
    g.set_state(U)
    g.set_ionosphere(**CFG)
    o = make_oracle(pr)
    o.set_state(U)
    moved = 0.0
    for _ in range(4):
        v, _, _ = I.couple(o.get_state(), pr.edges, pr.bc.dipole_moment, pr.bc.r_inner, oracle_cfg())
        moved = max(moved, np.abs(v).max())
        o.set_inner_velocity(v)
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    assert moved > 0
    assert np.max(rel_l1(g.get_state(), o.get_state())) <= MIXED_TOL


def test_form_bounds():
    pr = periodic_random((20, 12, 10), 2)
    g = make_gpu(pr, MIX)
    for axis, C in [(3, 5), (-1, 5), (0, 0), (0, 21)]:
        with pytest.raises(ppmlr.PPMLRError):
            g.set_march_chunk(axis, C)
    f = make_gpu(pr, ppmlr.PPMLR_FP64)
    assert f.set_sweep_form(0, 3, raise_on_error=False) == ppmlr.PPMLR_E_INVALID
