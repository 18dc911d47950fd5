"""Failure detection, made on the host: a NaN written into the state, a time
step far above the CFL limit, invalid arguments.  The kernels raise flags that
the next synchronising call reports; nothing traps or hangs."""
import numpy as np
import pytest

from gpu_util import make_gpu
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_MIXED])
@pytest.mark.parametrize("var,value", [(7, np.nan), (0, np.nan), (4, np.inf), (3, -np.inf)])
def test_nonfinite_state_reported(precision, var, value):
    # a non-finite total energy, density, normal field (B_x: the x sweep does
    # not update it) or transverse momentum in one cell
    pr = inputs.brio_wu_3d((16, 8, 8))
    U = pr.U0.copy()
    U[var, 3, 4, 5] = value
    g = ppmlr.Context.from_problem(pr, precision)
    g.set_state(U)
    g.step(1e-3)
    assert g.check(raise_on_error=False) == ppmlr.PPMLR_E_NONFINITE
    assert g.check(raise_on_error=False) == ppmlr.PPMLR_OK          # reported once


def test_cfl_violation_reported():
    pr = inputs.brio_wu_3d((16, 8, 8))
    g = make_gpu(pr)
    dt = g.cfl_dt(0.4)
    g.step(40 * dt)
    assert g.check(raise_on_error=False) in (ppmlr.PPMLR_E_CFL, ppmlr.PPMLR_E_NONFINITE)


def test_invalid_arguments():
    pr = inputs.brio_wu_3d((16, 8, 8))
    g = make_gpu(pr)
    assert g.step(-1.0, raise_on_error=False) == ppmlr.PPMLR_E_INVALID
    assert g.step(float("nan"), raise_on_error=False) == ppmlr.PPMLR_E_INVALID
    with pytest.raises(ppmlr.PPMLRError):
        g.sweep(3, 1e-3)
    with pytest.raises(ppmlr.PPMLRError):
        g.step_cfl(-0.4, 1)


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_FP64_EXACT])
def test_cfl_skips_a_nonfinite_cell_like_the_oracle(precision):
    """The CFL reduction ignores a cell whose state is NaN (the oracle's
    comparison does); the flag for the NaN comes from the sweep that made it."""
    from gpu_util import make_oracle
    pr = inputs.brio_wu_3d((16, 8, 8))
    U = pr.U0.copy()
    U[7, 3, 4, 5] = np.nan
    o = make_oracle(pr)
    o.set_state(U)
    g = ppmlr.Context.from_problem(pr, precision)
    g.set_state(U)
    dt_o, dt_g = o.cfl_dt(0.4), g.cfl_dt(0.4)
    assert np.isfinite(dt_g) and abs(dt_g - dt_o) <= 1e-14 * dt_o


def test_bounded_wait_gives_up_and_reports_timeout():
    """A device wait that nothing completes gives up after its bound: the
    timeout status is reported once and the context keeps working."""
    pr = inputs.brio_wu_3d((16, 8, 8))
    g, ref = make_gpu(pr), make_gpu(pr)
    g.selftest_wait_timeout()
    assert g.check(raise_on_error=False) == ppmlr.PPMLR_E_TIMEOUT
    assert g.check(raise_on_error=False) == ppmlr.PPMLR_OK
    for c in (g, ref):
        c.step_cfl(0.4, 3)
        c.check()
    assert np.array_equal(g.get_state(), ref.get_state())
