"""Pins for the oracle's nonlinear (two-shock, fast-mode) Riemann solver.

Fixed independently of the oracle: with B = 0 and two shocks the two-shock
solution is the exact gas-dynamic Riemann solution (computed by the separate
exact solver in exact_riemann.py); the Newton iteration converges
quadratically to it; the result lies on both shock curves for any states;
weak jumps reduce it to the two-wave solver to second order; uniform states
and mirror images behave as the physics requires; and the whole scheme with
the nonlinear solver converges on Sod's problem and holds the exact
post-shock plateau of a strong colliding-flow problem."""
import math

import numpy as np
import pytest

import oracle
from exact_riemann import sample, star_state
from paper_1607_02214_gb300 import inputs


def gas(rho, u, p):
    return [rho, u, 0.0, 0.0, 0.0, 0.0, p]


@pytest.mark.parametrize("g", [5.0 / 3.0, 1.4])
@pytest.mark.parametrize("case", [(1.0, 0.5, 1.0, 0.5, -0.5, 1.0), (1.0, 2.0, 1.0, 0.5, -2.0, 1.0),
                                  (1.0, 10.0, 1.0, 0.5, -10.0, 1.0), (2.0, 1.5, 3.0, 0.7, -1.0, 0.4)])
def test_two_shocks_match_the_exact_solution(g, case):
    rl, ul, pl, rr, ur, pr = case
    ps, us = star_state((rl, ul, pl), (rr, ur, pr), g)
    assert ps > max(pl, pr)                         # both waves are shocks
    o = oracle.riemann(gas(rl, ul, pl), gas(rr, ur, pr), 0.0, g, iters=8)
    assert o[1] == pytest.approx(ps, rel=1e-12)
    assert o[0] == pytest.approx(us, rel=1e-11, abs=1e-12)
    assert o[2] == o[1]                             # S* = P* without a normal field


def test_newton_converges_quadratically():
    g = 5.0 / 3.0
    ps, _ = star_state((1.0, 2.0, 1.0), (0.5, -2.0, 1.0), g)
    err = [abs(oracle.riemann(gas(1.0, 2.0, 1.0), gas(0.5, -2.0, 1.0), 0.0, g, iters=k)[1] / ps - 1)
           for k in range(5)]
    assert err[0] > 0.1                             # the two-wave start is far off for this strong pair
    assert err[2] < 2e-3 and err[3] < 2e-6 and err[4] < 1e-11
    for k in range(1, 4):
        assert err[k + 1] <= 10.0 * err[k] ** 2 / err[0] + 1e-15


def shock_speed(s, P, Bn, g):
    C = s[0] * math.sqrt(oracle.fast_speed2(s[0], s[6], Bn, s[4], s[5], g))
    Ps = s[6] + 0.5 * (s[4] ** 2 + s[5] ** 2)
    return C * math.sqrt(1.0 + (g + 1.0) / (2.0 * g) * (max(P, 0.0) / Ps - 1.0)), Ps


@pytest.mark.parametrize("seed", range(6))
def test_result_lies_on_both_shock_curves(seed):
    rng = np.random.default_rng(40 + seed)
    g = 5.0 / 3.0
    L = [rng.uniform(0.5, 2.0), rng.normal(), rng.normal(), rng.normal(), rng.normal(), rng.normal(),
         rng.uniform(0.5, 2.0)]
    R = [rng.uniform(0.5, 2.0), rng.normal(), rng.normal(), rng.normal(), rng.normal(), rng.normal(),
         rng.uniform(0.5, 2.0)]
    Bn = rng.normal()
    o = oracle.riemann(L, R, Bn, g, iters=30)
    us, Ps = o[0], o[1]
    WL, PL = shock_speed(L, Ps, Bn, g)
    WR, PR = shock_speed(R, Ps, Bn, g)
    assert us == pytest.approx(L[1] - (Ps - PL) / WL, rel=1e-12, abs=1e-12)
    assert us == pytest.approx(R[1] + (Ps - PR) / WR, rel=1e-12, abs=1e-12)
    assert o[2] == pytest.approx(Ps - 0.5 * Bn * Bn, rel=1e-14, abs=1e-14)
    lin = oracle.riemann(L, R, Bn, g)
    np.testing.assert_array_equal(o[3:7], lin[3:7])   # the Alfven subsystem is unchanged


def test_weak_jumps_reduce_to_the_two_wave_solver():
    g = 5.0 / 3.0
    base = [1.2, 0.3, -0.4, 0.2, 0.6, -0.5, 0.9]
    d = np.array([0.3, -0.5, 0.2, 0.1, -0.4, 0.3, 0.6])
    gaps = []
    for eps in (1e-2, 1e-3):
        L = list(np.array(base) - eps * d)
        R = list(np.array(base) + eps * d)
        nl = oracle.riemann(L, R, 0.7, g, iters=4)
        lin = oracle.riemann(L, R, 0.7, g)
        gaps.append(abs(nl[1] - lin[1]))
    assert gaps[1] < gaps[0] / 50.0                 # second order in the jump


def test_uniform_state_mirror_symmetry_and_zero_iterations():
    g = 5.0 / 3.0
    s = [1.3, 0.4, -0.2, 0.7, 0.5, -0.9, 0.8]
    o = oracle.riemann(s, s, 0.6, g, iters=4)
    assert o[0] == pytest.approx(s[1], abs=1e-15)
    assert o[1] == pytest.approx(s[6] + 0.5 * (s[4] ** 2 + s[5] ** 2), abs=1e-15)
    rng = np.random.default_rng(7)
    L = [1.4, 0.8, 0.1, -0.3, 0.4, 0.2, 1.1]
    R = [0.6, -0.9, 0.5, 0.2, -0.3, 0.6, 0.4]
    a = oracle.riemann(L, R, 0.5, g, iters=4)
    mL = list(R); mL[1] = -R[1]
    mR = list(L); mR[1] = -L[1]
    b = oracle.riemann(mL, mR, -0.5, g, iters=4)
    np.testing.assert_allclose(b[[0, 5, 6, 7]], -a[[0, 5, 6, 7]], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(b[[1, 2, 3, 4]], a[[1, 2, 3, 4]], rtol=1e-12, atol=1e-13)
    for _ in range(3):
        L = list(rng.uniform(0.5, 2.0, 7))
        R = list(rng.uniform(0.5, 2.0, 7))
        np.testing.assert_array_equal(oracle.riemann(L, R, 0.3, g, iters=0), oracle.riemann(L, R, 0.3, g))


def run_tube(pr, iters, t_end):
    from gpu_util import make_oracle
    o = make_oracle(pr)
    o.set_riemann(iters)
    _, _, flags = o.run(pr.cfl, t_end=t_end)
    assert flags == 0
    return o.get_state().reshape(8, -1)


def test_scheme_converges_on_sod_with_the_nonlinear_solver():
    g = 1.4
    errs = []
    for n in (100, 200, 400):
        U = run_tube(inputs.sod(n, gamma=g), 4, 0.2)
        xc = (np.arange(n) + 0.5) / n
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (xc - 0.5) / 0.2)
        errs.append(np.mean(np.abs(U[0] - ex[0])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.006
    order = math.log(errs[0] / errs[2], 4.0)
    assert order > 0.6, errs


def test_strong_colliding_flow_holds_the_exact_plateau():
    g = 5.0 / 3.0
    n = 400
    U = run_tube(inputs.shock_tube_1d(n, (1.0, 3.0, 0, 0, 0, 0, 0, 1.0), (1.0, -3.0, 0, 0, 0, 0, 0, 1.0), g),
                 4, 0.1)
    rho, m, E = U[0], U[1], U[7]
    p = (g - 1.0) * (E - 0.5 * m * m / rho)
    ps, us = star_state((1.0, 3.0, 1.0), (1.0, -3.0, 1.0), g)
    mid = slice(n // 2 - 10, n // 2 + 10)
    assert np.mean(p[mid]) == pytest.approx(ps, rel=1e-3)
    assert np.max(np.abs(m[mid])) < 1e-3 * ps
    # away from the wall-heating zone the density plateau is the shock-jump value
    rs = (ps + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps + 1)
    side = np.r_[n // 2 - 40:n // 2 - 20, n // 2 + 20:n // 2 + 40]
    assert np.mean(rho[side]) == pytest.approx(rs, rel=5e-3)
