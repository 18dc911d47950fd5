"""Ionosphere shell on the GPU against the oracle's (oracle/ionosphere.py):
the radial current and the cap potential from the same state, coupled steps
(FP64 to 1e-11, mixed to 1e-5), graph replay equal to direct steps bit for bit,
switching the shell off, invalid configurations, and the solve on the
256x192x192 magnetosphere state."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle, rel_l1
from oracle import ionosphere as I
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

CFG = dict(r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=16, n_phi=32)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def oracle_cfg(**kw):
    c = dict(CFG, **kw)
    return I.IonoConfig(c["r_iono"], c["r_fac"], c["sigma_p"], c["n_theta"], c["n_phi"])


def small():
    return inputs.magnetosphere(n=(48, 40, 36), h0=1.0)


def developed_state(pr, steps=6):
    """A state with field-aligned currents: a few FP64 steps from the initial
    condition (computed on the GPU; both sides then start from it)."""
    g = make_gpu(pr)
    g.run(pr.cfl, steps, graph_steps=0)
    return g.get_state()


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_current_and_potential_match_the_oracle():
    pr = small()
    U = developed_state(pr)
    g = make_gpu(pr)
    g.set_state(U)
    g.set_ionosphere(**CFG)
    g.ionosphere_solve()
    phi_g, jr_g = g.get_ionosphere()
    cfg = oracle_cfg()
    jr_o = I.radial_current(U, pr.edges, pr.bc.dipole_moment, pr.bc.r_inner, cfg)
    phi_o = I.solve_potential(jr_o, pr.bc.r_inner, cfg)
    assert np.abs(jr_o).max() > 0 and np.abs(phi_o).max() > 0
    assert rel_max(jr_g, jr_o) <= 1e-11, rel_max(jr_g, jr_o)
    assert rel_max(phi_g, phi_o) <= 1e-11, rel_max(phi_g, phi_o)


def coupled_pair(pr, U, precision, nsteps, cfg_kw=None):
    kw = dict(CFG, **(cfg_kw or {}))
    o = make_oracle(pr)
    o.set_state(U)
    g = make_gpu(pr, precision)
    g.set_state(U)
    g.set_ionosphere(**kw)
    cfg = oracle_cfg(**(cfg_kw or {}))
    moved = 0.0
    for _ in range(nsteps):
        v, _, _ = I.couple(o.get_state(), pr.edges, pr.bc.dipole_moment, pr.bc.r_inner, cfg)
        moved = max(moved, np.abs(v).max())
        o.set_inner_velocity(v)
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    return o, g, moved


@pytest.mark.parametrize("precision,tol", [(ppmlr.PPMLR_FP64, 1e-11), (ppmlr.PPMLR_FP64_EXACT, 1e-11),
                                           (ppmlr.PPMLR_MIXED, 1e-5)])
def test_coupled_steps_match_the_oracle(precision, tol):
    pr = small()
    U = developed_state(pr)
    o, g, moved = coupled_pair(pr, U, precision, 5)
    assert moved > 0.0                               # the shell drives the inner cells
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= tol, err


def test_coupled_steps_other_grid_and_cap_resolution():
    pr = inputs.magnetosphere(n=(56, 44, 40), h0=0.8)
    U = developed_state(pr, 4)
    o, g, moved = coupled_pair(pr, U, ppmlr.PPMLR_FP64, 3, dict(n_theta=7, n_phi=10, r_fac=3.5, sigma_p=2.0))
    assert moved > 0.0
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= 1e-11, err


def test_graph_replay_equals_direct_steps_with_the_shell():
    pr = small()
    U = developed_state(pr, 2)
    a, b = make_gpu(pr), make_gpu(pr)
    for c in (a, b):
        c.set_state(U)
        c.set_ionosphere(**CFG)
    a.run(pr.cfl, 8, graph_steps=4)
    b.run(pr.cfl, 8, graph_steps=0)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.time == b.time


def test_shell_off_restores_the_fixed_inner_state():
    pr = small()
    U = developed_state(pr, 2)
    a, b = make_gpu(pr), make_gpu(pr)
    for c in (a, b):
        c.set_state(U)
    a.set_ionosphere(**CFG)
    a.run(pr.cfl, 2, graph_steps=2)
    a.set_ionosphere(on=False)
    a.set_state(U)
    a.set_step_count(0)
    b.run(pr.cfl, 2, graph_steps=2)
    a.run(pr.cfl, 2, graph_steps=2)
    assert np.array_equal(a.get_state(), b.get_state())
    with pytest.raises(ppmlr.PPMLRError):
        a.ionosphere_solve()


def test_invalid_configurations_are_refused():
    pr = small()
    g = make_gpu(pr)
    for bad in (dict(r_fac=200.0), dict(r_iono=3.5), dict(n_phi=33), dict(n_theta=1), dict(sigma_p=0.0),
                dict(r_fac=0.5)):
        with pytest.raises(ppmlr.PPMLRError):
            g.set_ionosphere(**dict(CFG, **bad))
    with pytest.raises(ppmlr.PPMLRError):
        g.ionosphere_solve()                         # still off
    tube = make_gpu(inputs.brio_wu_3d((16, 16, 16)))   # no inner sphere, no dipole
    with pytest.raises(ppmlr.PPMLRError):
        tube.set_ionosphere(**CFG)


def test_solve_on_the_full_magnetosphere_grid():
    pr = inputs.magnetosphere(n=(256, 192, 192), h0=0.4)
    g = make_gpu(pr)
    g.run(pr.cfl, 4, graph_steps=0)
    U = g.get_state()
    g.set_ionosphere(r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=24, n_phi=48)
    g.ionosphere_solve()
    phi_g, jr_g = g.get_ionosphere()
    cfg = I.IonoConfig(1.017, 4.0, 0.6283, 24, 48)
    jr_o = I.radial_current(U, pr.edges, pr.bc.dipole_moment, pr.bc.r_inner, cfg)
    phi_o = I.solve_potential(jr_o, pr.bc.r_inner, cfg)
    assert rel_max(jr_g, jr_o) <= 1e-11 and rel_max(phi_g, phi_o) <= 1e-11


def test_before_the_first_solve_the_inner_cells_keep_the_fixed_state():
    """A lone sweep right after the shell is switched on (no step, no solve)
    equals the sweep without the shell, bit for bit."""
    pr = small()
    U = developed_state(pr, 2)
    a, b = make_gpu(pr), make_gpu(pr)
    for c in (a, b):
        c.set_state(U)
    a.set_ionosphere(**CFG)
    for axis in (0, 1, 2):
        a.sweep(axis, 1e-3)
        b.sweep(axis, 1e-3)
    assert np.array_equal(a.get_state(), b.get_state())
