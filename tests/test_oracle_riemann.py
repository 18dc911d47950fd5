"""Pins for the oracle's linearised Lagrangian MHD Riemann solver and wave speeds."""
import math

import numpy as np
import pytest

import oracle
from exact_riemann import star_state

G53 = 5.0 / 3.0


def rand_state(rng):
    return [rng.uniform(0.5, 2.0), rng.normal(), rng.normal(), rng.normal(),
            rng.normal(), rng.normal(), rng.uniform(0.5, 2.0)]


def test_uniform_state_is_reproduced():
    s = [1.3, 0.4, -0.2, 0.7, 0.5, -0.9, 0.8]
    Bn = 0.6
    o = oracle.riemann(s, s, Bn, G53)
    P = s[6] + 0.5 * (s[4] ** 2 + s[5] ** 2)
    assert o[0] == pytest.approx(s[1], abs=1e-15)
    assert o[1] == pytest.approx(P, abs=1e-15)
    assert o[2] == pytest.approx(P - 0.5 * Bn * Bn, abs=1e-15)
    assert o[3] == pytest.approx(s[2], abs=1e-15) and o[4] == pytest.approx(s[3], abs=1e-15)
    assert o[5] == pytest.approx(Bn * s[4], abs=1e-15) and o[6] == pytest.approx(Bn * s[5], abs=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_mirror_symmetry(seed):
    # Reflecting the normal axis swaps the sides, flips u and B_n (so sigma),
    # keeps P and v_t: u* -> -u*, P* same, v* same, sigma* -> -sigma*, F_E -> -F_E.
    rng = np.random.default_rng(seed)
    L, R = rand_state(rng), rand_state(rng)
    Bn = rng.normal()
    a = oracle.riemann(L, R, Bn, G53)
    mL = list(R); mL[1] = -R[1]
    mR = list(L); mR[1] = -L[1]
    b = oracle.riemann(mL, mR, -Bn, G53)
    np.testing.assert_allclose(b[[0, 5, 6, 7]], -a[[0, 5, 6, 7]], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(b[[1, 2, 3, 4]], a[[1, 2, 3, 4]], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_riemann_invariants_hold(seed):
    # The solution is where the two incoming invariants meet:
    #   P* - P_L = -W_L (u* - u_L),   P* - P_R = W_R (u* - u_R)
    #   s* - Z_L v* = s_L - Z_L v_L,   s* + Z_R v* = s_R + Z_R v_R
    rng = np.random.default_rng(10 + seed)
    L, R = rand_state(rng), rand_state(rng)
    Bn = rng.normal()
    o = oracle.riemann(L, R, Bn, G53)
    us, Ps = o[0], o[1]
    W = lambda s: s[0] * math.sqrt(oracle.fast_speed2(s[0], s[6], Bn, s[4], s[5], G53))
    P = lambda s: s[6] + 0.5 * (s[4] ** 2 + s[5] ** 2)
    assert Ps - P(L) == pytest.approx(-W(L) * (us - L[1]), rel=1e-12, abs=1e-13)
    assert Ps - P(R) == pytest.approx(W(R) * (us - R[1]), rel=1e-12, abs=1e-13)
    ZL, ZR = math.sqrt(L[0]) * abs(Bn), math.sqrt(R[0]) * abs(Bn)
    for t in range(2):
        v, s = o[3 + t], o[5 + t]
        assert s - ZL * v == pytest.approx(Bn * L[4 + t] - ZL * L[2 + t], rel=1e-12, abs=1e-13)
        assert s + ZR * v == pytest.approx(Bn * R[4 + t] + ZR * R[2 + t], rel=1e-12, abs=1e-13)
    assert o[7] == pytest.approx(o[2] * o[0] - o[5] * o[3] - o[6] * o[4], rel=1e-14, abs=1e-14)


def test_zero_normal_field():
    L = [1.0, 0.1, 0.3, -0.2, 0.4, 0.5, 1.0]
    R = [0.5, -0.2, -0.1, 0.6, -0.3, 0.2, 0.4]
    o = oracle.riemann(L, R, 0.0, G53)
    assert o[5] == 0.0 and o[6] == 0.0
    assert o[3] == pytest.approx(0.5 * (L[2] + R[2])) and o[4] == pytest.approx(0.5 * (L[3] + R[3]))


@pytest.mark.parametrize("eps", [1e-2, 5e-3, 2.5e-3])
def test_acoustic_limit_matches_exact_gas_solver_to_second_order(eps):
    # With B = 0 the normal subsystem is the linearised gas-dynamics solver.
    # For a jump of size eps its star state differs from the exact Riemann
    # solution by O(eps^2).
    g = 1.4
    L = [1.0, 0.0, 0, 0, 0, 0, 1.0]
    R = [1.0 - eps, -eps, 0, 0, 0, 0, 1.0 - 1.3 * eps]
    o = oracle.riemann(L, R, 0.0, g)
    p_ex, u_ex = star_state((L[0], L[1], L[6]), (R[0], R[1], R[6]), g)
    assert abs(o[1] - p_ex) < 0.5 * eps ** 2
    assert abs(o[0] - u_ex) < 0.5 * eps ** 2


def test_fast_speed_closed_forms():
    g = G53
    rho, p = 1.7, 0.9
    a2 = g * p / rho
    # no normal field: c_f^2 = a^2 + b^2
    assert oracle.fast_speed2(rho, p, 0.0, 0.6, -0.8, g) == pytest.approx(a2 + 1.0 / rho, rel=1e-14)
    # field purely normal: c_f = max(a, b_n)
    for Bn in (0.3, 3.0):
        assert oracle.fast_speed2(rho, p, Bn, 0.0, 0.0, g) == pytest.approx(max(a2, Bn * Bn / rho), rel=1e-14)
    # no field: sound speed
    assert oracle.fast_speed2(rho, p, 0.0, 0.0, 0.0, g) == pytest.approx(a2, rel=1e-15)


def test_dipole_field_properties():
    M = 6543.6
    # equator: B = +M / r^3 along z; pole: B = -2 M / r^3 along z (moment along -z)
    np.testing.assert_allclose(oracle.dipole(M, 3.0, 0.0, 0.0), [0, 0, M / 27.0], rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(oracle.dipole(M, 0.0, 0.0, 4.0), [0, 0, -2 * M / 64.0], rtol=1e-14, atol=1e-12)
    # divergence- and curl-free away from the origin (central differences)
    rng = np.random.default_rng(3)
    h = 1e-4
    for _ in range(20):
        x = rng.uniform(-8, 8, size=3)
        if np.linalg.norm(x) < 2:
            continue
        J = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            J[:, k] = (oracle.dipole(M, *(x + e)) - oracle.dipole(M, *(x - e))) / (2 * h)
        scale = np.linalg.norm(oracle.dipole(M, *x)) / np.linalg.norm(x)
        assert abs(np.trace(J)) < 1e-6 * scale
        assert np.max(np.abs(J - J.T)) < 1e-6 * scale
    # the image dipole at (30, 0, 0) cancels B_x on the plane x = 15
    for y, z in [(3.0, 4.0), (-7.0, 2.5), (0.0, -9.0)]:
        bx = oracle.dipole(M, 15.0, y, z)[0] + oracle.dipole(M, 15.0 - 30.0, y, z)[0]
        assert abs(bx) < 1e-12 * M
