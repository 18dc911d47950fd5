"""Pins for the oracle's contact steepening in the remap (Colella & Woodward
1984 discontinuity detection, applied with one weight to all seven remapped
densities).

Fixed independently of the oracle: an advected contact (density jump with
uniform velocity and pressure) stays sharper than without steepening while
velocity and pressure stay uniform (every remapped density is affine in the
density across a contact, so one weight keeps them consistent); a smooth,
well-resolved density wave is not touched at all (bit-identical run); Sod's
problem gets closer to the exact solution; the strong colliding flow keeps
its exact plateau."""
import numpy as np
import pytest

from exact_riemann import sample, star_state
from gpu_util import make_oracle
from paper_1607_02214_gb300 import inputs

G53 = 5.0 / 3.0


def run(pr, steepen, t_end):
    o = make_oracle(pr)
    o.set_steepening(steepen)
    _, k, flags = o.run(pr.cfl, t_end=t_end)
    assert flags == 0
    return o.get_state().reshape(8, -1), k


def advected_contact(n):
    return inputs.shock_tube_1d(n, (1.0, 1.0, 0, 0, 0, 0, 0, 1.0), (0.125, 1.0, 0, 0, 0, 0, 0, 1.0), G53,
                                periodic=True)


def width(rho, lo=0.125, hi=1.0):
    return int(((rho > lo + 0.1 * (hi - lo)) & (rho < hi - 0.1 * (hi - lo))).sum())


def test_contact_stays_sharp_and_in_pressure_balance():
    widths = []
    for steepen in (0, 1):
        U, _ = run(advected_contact(200), steepen, 0.3)
        rho = U[0]
        u = U[1] / rho
        p = (G53 - 1.0) * (U[7] - 0.5 * U[1] ** 2 / rho)
        assert np.max(np.abs(p - 1.0)) < 1e-7
        assert np.max(np.abs(u - 1.0)) < 1e-7
        widths.append(width(rho))
    assert widths[1] <= 5 and widths[1] * 2 <= widths[0], widths


def test_smooth_wave_is_left_alone():
    n = 200
    pr = inputs.shock_tube_1d(n, (1.0, 1.0, 0, 0, 0, 0, 0, 1.0), (1.0, 1.0, 0, 0, 0, 0, 0, 1.0), G53, periodic=True)
    e = inputs.uniform_axis(n, 0.0, 1.0)
    rho = 1.0 + 0.5 * (np.cos(2 * np.pi * e[:-1]) - np.cos(2 * np.pi * e[1:])) / (2 * np.pi * np.diff(e))
    one, zero = np.ones(n), np.zeros(n)
    pr.U0[:] = inputs.conserved(rho, (one, zero, zero), (zero, zero, zero), one, G53).reshape(pr.U0.shape)
    a, _ = run(pr, 0, 0.2)
    b, _ = run(pr, 1, 0.2)
    assert np.array_equal(a, b)


def test_sod_gets_closer_to_the_exact_solution():
    n, g = 400, 1.4
    xc = (np.arange(n) + 0.5) / n
    ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (xc - 0.5) / 0.2)
    errs = []
    for steepen in (0, 1):
        U, _ = run(inputs.sod(n, gamma=g), steepen, 0.2)
        errs.append(np.mean(np.abs(U[0] - ex[0])))
    assert errs[1] < 0.9 * errs[0], errs


def test_strong_colliding_flow_keeps_its_plateau():
    n = 400
    U, _ = run(inputs.shock_tube_1d(n, (1.0, 3.0, 0, 0, 0, 0, 0, 1.0), (1.0, -3.0, 0, 0, 0, 0, 0, 1.0), G53), 1, 0.1)
    rho, m, E = U[0], U[1], U[7]
    p = (G53 - 1.0) * (E - 0.5 * m * m / rho)
    ps, _ = star_state((1.0, 3.0, 1.0), (1.0, -3.0, 1.0), G53)
    assert np.mean(p[n // 2 - 10:n // 2 + 10]) == pytest.approx(ps, rel=1e-3)
