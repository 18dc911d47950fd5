"""Parity on a developed magnetosphere state.

The initial state of Sec. IV-A is mostly quiescent: a whole-grid L1 over a
few steps is dominated by the undisturbed solar wind and the field-free
region, and local errors at the forming shock and near the dipole are
diluted.  Here the oracle advances the 96x72x72 magnetosphere (the
256x192x192 extent at 0.4 * 256 / 96 R_E resolution, dipole, inner sphere
r = 3 R_E, solar-wind inflow) for 400 steps of its own CFL time step: the
wind's shock compresses the plasma to nearly twice the wind density, the
field perturbation near the dipole grows until thousands of cells sit at the
pressure floor, and over a hundred cells between the inner sphere and 8 R_E
have plasma beta below 0.01.  Every GPU form replays the same time steps
from the same initial state and is compared cell by cell at the end with the
strict per-variable relative L1 (sum |a - b| / sum |b| per variable): the
exact FP64 form bit for bit, the contracted FP64 form within 1e-11, the
mixed form within 1e-5, except the weak transverse momenta (their sums are
~1e-3 of the momentum's), whose strict figure is held to 1e-4 and their
group-scaled figure to 1e-5.  For the mixed form (FP32 reconstruction, Riemann
solve and remap; pressure recovered in double-float arithmetic) the pressure
recovered from the final state in the cells between the inner sphere and
8 R_E is compared with the oracle's: its difference, relative to the cell's
total energy density (the scale of the cancellation E - rho v^2/2 -
|B'|^2/2), is bounded.
"""
import numpy as np
import pytest

from gpu_util import assert_parity, linf, make_gpu, make_oracle, rel_l1, rel_l1_group
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

GRID = (96, 72, 72)
H0 = 0.4 * 256 / 96
NSTEPS = 400
# mixed form: pressure difference in 3 < r < 8 R_E relative to the local
# total energy density -- after 400 steps (mean and worst cell) and after one
# sweep from the oracle's developed state
MIXED_P_MEAN_TOL = 1e-5
MIXED_P_MAX_TOL = 2e-3
MIXED_P_SWEEP_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def developed():
    pr = inputs.magnetosphere(n=GRID, h0=H0)
    o = make_oracle(pr)
    dts = []
    for _ in range(NSTEPS):
        dt = o.cfl_dt(pr.cfl)
        dts.append(dt)
        assert o.step(dt) == 0
    return pr, dts, o.get_state(), o.floor_hits


def pressure(U, gamma):
    return (gamma - 1.0) * (U[7] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
                            - 0.5 * (U[4] ** 2 + U[5] ** 2 + U[6] ** 2))


def radius(pr):
    c = [0.5 * (e[1:] + e[:-1]) for e in pr.edges]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return np.sqrt(x * x + y * y + z * z)


def test_the_state_is_developed(developed):
    pr, dts, U, floors = developed
    rho_sw = pr.bc.inflow[0]
    r = radius(pr)
    beta = pressure(U, pr.gamma) / np.maximum(0.5 * (U[4] ** 2 + U[5] ** 2 + U[6] ** 2), 1e-300)
    shell = (r > pr.bc.r_inner) & (r < 8.0)
    assert np.all(np.isfinite(U))
    assert U[0].max() > 1.5 * rho_sw                  # shock compression
    assert floors > 1000                              # the pressure floor is in use
    assert np.count_nonzero(shell & (beta < 0.01)) > 50   # low-beta cells near the dipole


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
def test_developed_parity(developed, precision):
    pr, dts, ref, floors = developed
    g = make_gpu(pr, precision)
    g.autotune()                                      # the launch forms the benchmark times
    for dt in dts:
        g.step(dt)
    g.check()
    a = g.get_state()
    err, errg, inf = rel_l1(a, ref), rel_l1_group(a, ref), linf(a, ref)
    print(f"\nprecision {precision}: rel L1 {err}\n  group-scaled {errg}\n  Linf {inf}"
          f"\n  floors {g.diagnostics()['floor_hits']} (oracle {floors})")
    if precision == ppmlr.PPMLR_FP64_EXACT:
        assert np.array_equal(a, ref)
        assert g.diagnostics()["floor_hits"] == floors
    elif precision == ppmlr.PPMLR_FP64:
        assert np.max(err) <= 1e-11, err
    else:
        # strict per-variable 1e-5; the weak transverse momenta (sums ~1e-3
        # of the momentum's) 1e-4 strict and 1e-5 group-scaled
        assert_parity(a, ref, 1e-5, 1e-4)
        r = radius(pr)
        shell = (r > pr.bc.r_inner) & (r < 8.0)
        dp = np.abs(pressure(a, pr.gamma) - pressure(ref, pr.gamma))[shell]
        scale = np.abs(ref[7])[shell]
        rel = dp / scale
        print(f"  pressure 3 < r < 8 after {NSTEPS} steps: |dp| / E max {rel.max():.3e}, "
              f"99.9 % {np.quantile(rel, 0.999):.3e}, mean {rel.mean():.3e}")
        # after 400 steps the FP32 drift of the state dominates (the worst cell
        # sits where the floor decision of the two paths differs)
        assert rel.mean() <= MIXED_P_MEAN_TOL and rel.max() <= MIXED_P_MAX_TOL


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mixed_pressure_one_sweep_from_the_developed_state(developed, axis):
    # One sweep of the mixed form and of the oracle from the oracle's
    # developed state: the pressure recovered from the output, in the cells
    # between the inner sphere and 8 R_E, relative to the total energy density.
    pr, dts, ref, _ = developed
    o = make_oracle(pr)
    o.set_state(ref)
    dt = o.cfl_dt(pr.cfl)
    assert o.sweep(axis, dt) == 0
    g = make_gpu(pr, ppmlr.PPMLR_MIXED)
    g.set_state(ref)
    g.sweep(axis, dt)
    g.check()
    a, b = g.get_state(), o.get_state()
    r = radius(pr)
    shell = (r > pr.bc.r_inner) & (r < 8.0)
    rel = np.abs(pressure(a, pr.gamma) - pressure(b, pr.gamma))[shell] / np.abs(b[7])[shell]
    print(f"\naxis {axis}: one sweep, pressure 3 < r < 8: |dp| / E max {rel.max():.3e}, mean {rel.mean():.3e}; "
          f"rel L1 {rel_l1(a, b)}")
    assert rel.max() <= MIXED_P_SWEEP_TOL
    assert_parity(a, b, 1e-5, 1e-4)
