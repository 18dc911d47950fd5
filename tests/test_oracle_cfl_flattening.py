"""Pins of the oracle's CFL time step and flattening coefficient against
values fixed by hand and by the mathematics, not by the oracle's own output.

* Flattening (Colella & Woodward 1984, App. A, cited by the paper's Sec. II
  for its PPM reconstruction; total pressure for MHD): pressure/velocity
  profiles whose shock test, steepness, clamp and low-pressure-side
  neighbour are worked out by hand at named zones.
* CFL (the step-size rule of the scheme's explicit update: the fastest
  signal may cross at most `cfl` of a zone per step): closed-form states on
  one- and two-cell grids where the dipole field decides the fast speed, the
  inner sphere is skipped and the pressure floor is used; and random states
  against the largest eigenvalue of the 1D ideal-MHD Jacobian computed by
  numpy.linalg.eigvals (|v_n| + c_f is the largest characteristic speed).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
with open(os.path.join(GOLD, "cw84_constants.json")) as fh:
    FL = json.load(fh)["flattening"]
EPS, W1, W2 = FL["epsilon"], FL["omega1"], FL["omega2"]


# ---------------------------------------------------------------- flattening

def _ft_by_hand(steep):
    return max(0.0, min(1.0, W2 * (steep - W1)))


def test_flattening_partial_shock_zone_and_low_pressure_neighbour():
    # Pressure rises to the right through zones 4..6; flow compressive.
    #   zone 5: jump Pt6 - Pt4 = 0.8 > EPS * 1.1, steepness 0.8 / (Pt7 - Pt3) = 0.8
    #           -> ft = 10 (0.8 - 0.75) = 0.5
    #   zone 4: jump 0.5 > EPS * 1.0 but steepness 0.5 / 0.9 < 0.75 -> 0
    #   zone 6: jump 0.5 > EPS * 1.5 = 0.495, steepness 0.5 / 0.9 -> 0
    #   zones 3 and 7: jump 0.1 < EPS -> no shock
    # Coefficient: pressure rises to the right, so each zone also takes the
    # indicator of its left (low-pressure) neighbour: f5 = 0.5 and f6 = 0.5,
    # f4 = f7 = 0.
    Pt = np.array([1.0, 1.0, 1.0, 1.0, 1.1, 1.5, 1.9, 2.0, 2.0, 2.0, 2.0])
    u = np.array([1.0, 1.0, 1.0, 1.0, 0.8, 0.5, 0.2, 0.0, 0.0, 0.0, 0.0])
    ft, f = oracle.flatten(Pt, u)
    assert ft[5] == pytest.approx(_ft_by_hand(0.8), abs=1e-12) and ft[5] == pytest.approx(0.5, abs=1e-12)
    np.testing.assert_array_equal(np.delete(ft, 5), 0.0)
    np.testing.assert_allclose(f[3:8], [0.0, 0.0, 0.5, 0.5, 0.0], atol=1e-12)

    # Mirror image (pressure rising to the left, flow still compressive):
    # the low-pressure side is now the right neighbour, so zones 5 and 4
    # (the mirror of 5 and 6) carry 0.5.
    ftm, fm = oracle.flatten(Pt[::-1].copy(), -u[::-1].copy())
    np.testing.assert_allclose(ftm, ft[::-1], atol=1e-12)
    np.testing.assert_allclose(fm[3:8], [0.0, 0.5, 0.5, 0.0, 0.0], atol=1e-12)


def test_flattening_threshold_epsilon():
    # A step in Pt across zone 3 with flat shoulders (steepness exactly 1,
    # ft clamped to 1 once detected); the relative jump just below and just
    # above EPS.
    for ratio, expect in ((EPS - 0.01, 0.0), (EPS + 0.01, 1.0)):
        Pt = np.array([1.0, 1.0, 1.0, 1.0 + ratio / 2, 1.0 + ratio, 1.0 + ratio, 1.0 + ratio])
        # zone 3: jump Pt4 - Pt2 = ratio, smaller neighbour 1.0, den Pt5 - Pt1 = ratio
        u = np.array([1.0, 1.0, 1.0, 0.5, 0.0, 0.0, 0.0])
        ft, f = oracle.flatten(Pt, u)
        assert ft[3] == pytest.approx(expect, abs=1e-12)
        assert f[3] == pytest.approx(expect, abs=1e-12)


def test_flattening_needs_compression():
    # The same profile as the partial-shock case with an expanding flow.
    Pt = np.array([1.0, 1.0, 1.0, 1.0, 1.1, 1.5, 1.9, 2.0, 2.0, 2.0, 2.0])
    u = -np.array([1.0, 1.0, 1.0, 1.0, 0.8, 0.5, 0.2, 0.0, 0.0, 0.0, 0.0])
    ft, f = oracle.flatten(Pt, u)
    assert not ft.any() and not f.any()


def test_flattening_vanishing_wide_difference_is_maximally_steep():
    # Zone 3: Pt2 = 1, Pt4 = 2 (jump 1 > EPS), Pt1 = Pt5 = 1.5 (wide
    # difference 0) -> steepness 1 -> ft = min(1, 10 * 0.25) = 1.
    Pt = np.array([1.5, 1.5, 1.0, 1.4, 2.0, 1.5, 1.5])
    u = np.array([0.0, 0.0, 1.0, 0.5, 0.0, 0.0, 0.0])
    ft, _ = oracle.flatten(Pt, u)
    assert ft[3] == pytest.approx(1.0, abs=1e-12)


def test_flattening_steepness_scale():
    # Steepness 0.78 and 0.8 and 0.85: ft = 0.3, 0.5, 1.0 (W2 scale, W1 offset).
    for steep, expect in ((0.78, 0.3), (0.8, 0.5), (0.85, 1.0)):
        jump = 0.8
        den = jump / steep
        # zone 3 (pencil of 7): Pt1, Pt5 at -den/2, +den/2 about 2; Pt2, Pt4 at -jump/2, +jump/2
        Pt = np.array([2 - den / 2, 2 - den / 2, 2 - jump / 2, 2.0, 2 + jump / 2, 2 + den / 2, 2 + den / 2])
        u = np.array([1.0, 1.0, 1.0, 0.5, 0.0, 0.0, 0.0])
        ft, _ = oracle.flatten(Pt, u)
        assert ft[3] == pytest.approx(expect, abs=1e-12), steep


# ---------------------------------------------------------------------- CFL

GAM = 5.0 / 3.0


def _cons(rho, v, Bp, p, gam=GAM):
    v = np.asarray(v, float)
    Bp = np.asarray(Bp, float)
    return np.array([rho, *(rho * v), *Bp, p / (gam - 1) + 0.5 * rho * v @ v + 0.5 * Bp @ Bp])


def _oracle(edges, M=0.0, r_inner=0.0, p_min=1e-12):
    return oracle.Oracle(edges, GAM, [oracle.BC_OUTFLOW] * 6, inflow=np.zeros(8), dipole_moment=M,
                         r_inner=r_inner, inner=np.array([1.0, 0, 0, 0, 0, 0, 0, 1.0]), p_min=p_min)


def test_cfl_closed_form_dipole_decides_fast_speed():
    # One cell centred at (2, 0, 0) on the dipole's equator, M = 8:
    # B_d = (0, 0, M / r^3) = (0, 0, 1).  rho = 1, p = 0.6 (a^2 = gamma p / rho
    # = 1), v = (2, 0, 0), B' = 0.  Along x: c_f(B') = 1, c_f(B' + B_d) = sqrt(a^2
    # + b^2) = sqrt(2) (field normal to x) -> dx / (2 + sqrt 2) with dx = 1.
    # Along y: 1 / sqrt 2.  Along z (field along z): c_f^2 = max(a^2, b^2) = 1,
    # dz = 0.5 -> 0.5.  dt = cfl / (2 + sqrt 2).
    o = _oracle([np.array([1.5, 2.5]), np.array([-0.5, 0.5]), np.array([-0.25, 0.25])], M=8.0)
    U = _cons(1.0, [2.0, 0.0, 0.0], [0.0, 0.0, 0.0], 0.6).reshape(8, 1, 1, 1)
    o.set_state(U)
    assert o.cfl_dt(0.4) == pytest.approx(0.4 / (2.0 + math.sqrt(2.0)), rel=1e-14)


def test_cfl_skips_inner_sphere_and_uses_both_fields():
    # Cell 0 centred at r = 0.5 inside r_inner = 1 with a huge velocity (its
    # bound would be tiny) is skipped; cell 1 at (2, 0, 0), width 2, v_x = 4,
    # B_d = (0, 0, 1): x bound 2 / (4 + sqrt 2), y 1 / sqrt 2, z 0.5.
    o = _oracle([np.array([0.0, 1.0, 3.0]), np.array([-0.5, 0.5]), np.array([-0.25, 0.25])], M=8.0,
                r_inner=1.0)
    U = np.stack([_cons(1.0, [1e6, 0, 0], [0, 0, 0], 0.6), _cons(1.0, [4.0, 0, 0], [0, 0, 0], 0.6)], axis=-1)
    o.set_state(U.reshape(8, 1, 1, 2))
    assert o.cfl_dt(0.5) == pytest.approx(0.5 * 2.0 / (4.0 + math.sqrt(2.0)), rel=1e-14)


def test_cfl_uses_the_perturbation_field_when_it_is_larger():
    # B' = (0, 3, 0) and B_d = (0, 0, 1): |B' + B_d|^2 = 10 > |B'|^2 = 9 along x
    # (both normal), so c_f^2 = 1 + 10; along y (B'_n = 3): c_f^2(B') = max(1, 9)
    # = 9 < c_f^2(B' + B_d) = (11 + sqrt(121 - 36)) / 2; along z: B' alone
    # gives 1 + 9 = 10 (normal field 0), B' + B_d (a^2 + b^2 = 11, bn^2 = 1)
    # gives (11 + sqrt(117)) / 2 = 10.9.
    o = _oracle([np.array([1.5, 2.5]), np.array([-0.5, 0.5]), np.array([-0.25, 0.25])], M=8.0)
    o.set_state(_cons(1.0, [0.0, 0.0, 0.0], [0.0, 3.0, 0.0], 0.6).reshape(8, 1, 1, 1))
    bx = 1.0 / math.sqrt(11.0)
    by = 1.0 / math.sqrt((11.0 + math.sqrt(121.0 - 36.0)) / 2.0)
    bz = 0.5 / math.sqrt(max(10.0, (11.0 + math.sqrt(117.0)) / 2.0))
    assert o.cfl_dt(1.0) == pytest.approx(min(bx, by, bz), rel=1e-14)


def test_cfl_pressure_floor():
    # E = kinetic energy only -> recovered p = 0 < p_min = 0.06, floored:
    # a^2 = gamma * 0.06 = 0.1; no field.  v = (0.5, 0, 0): bounds
    # 1 / (0.5 + sqrt 0.1), 1 / sqrt 0.1, 0.5 / sqrt 0.1.
    o = _oracle([np.array([1.5, 2.5]), np.array([-0.5, 0.5]), np.array([-0.25, 0.25])], p_min=0.06)
    o.set_state(_cons(1.0, [0.5, 0.0, 0.0], [0.0, 0.0, 0.0], 0.0).reshape(8, 1, 1, 1))
    a = math.sqrt(0.1)
    assert o.cfl_dt(1.0) == pytest.approx(min(1.0 / (0.5 + a), 0.5 / a), rel=1e-13)


def _max_char_speed(rho, v, B, p, d, gam=GAM):
    """Largest |eigenvalue| of the 1D ideal-MHD Jacobian along axis d in the
    primitive variables (rho, u, v1, v2, B1, B2, p), mu0 = 1."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    u, v1, v2 = v[d], v[t1], v[t2]
    Bn, B1, B2 = B[d], B[t1], B[t2]
    A = np.zeros((7, 7))
    A[0] = [u, rho, 0, 0, 0, 0, 0]
    A[1] = [0, u, 0, 0, B1 / rho, B2 / rho, 1 / rho]
    A[2] = [0, 0, u, 0, -Bn / rho, 0, 0]
    A[3] = [0, 0, 0, u, 0, -Bn / rho, 0]
    A[4] = [0, B1, -Bn, 0, u, 0, 0]
    A[5] = [0, B2, 0, -Bn, 0, u, 0]
    A[6] = [0, gam * p, 0, 0, 0, 0, u]
    return np.max(np.abs(np.linalg.eigvals(A)))


def _dipole(M, x, y, z):
    r2 = x * x + y * y + z * z
    r5 = r2 ** 2.5
    mr = -z                                   # moment along -z
    return np.array([M * 3 * mr * x / r5, M * 3 * mr * y / r5, M * (3 * mr * z + r2) / r5])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cfl_random_states_against_jacobian_eigenvalues(seed):
    rng = np.random.default_rng(seed)
    n = (5, 4, 3)
    edges = [np.cumsum(np.r_[lo, rng.uniform(0.3, 1.2, k)]) for lo, k in zip((-3.1, -2.2, -1.7), n)]
    M, r_inner = 4.0, 1.3
    o = _oracle(edges, M=M, r_inner=r_inner, p_min=1e-9)
    U = np.zeros((8, n[2], n[1], n[0]))
    best = np.inf
    for iz in range(n[2]):
        for iy in range(n[1]):
            for ix in range(n[0]):
                rho = rng.uniform(0.5, 2.0)
                v = rng.normal(0, 1.0, 3)
                Bp = rng.normal(0, 1.0, 3)
                p = rng.uniform(0.1, 1.0)
                U[:, iz, iy, ix] = _cons(rho, v, Bp, p)
                c = [0.5 * (edges[d][i] + edges[d][i + 1]) for d, i in enumerate((ix, iy, iz))]
                if c[0] ** 2 + c[1] ** 2 + c[2] ** 2 < r_inner ** 2:
                    continue
                Bd = _dipole(M, *c)
                for d, i in enumerate((ix, iy, iz)):
                    s = max(_max_char_speed(rho, v, Bp, p, d), _max_char_speed(rho, v, Bp + Bd, p, d))
                    best = min(best, (edges[d][i + 1] - edges[d][i]) / s)
    o.set_state(U)
    assert o.cfl_dt(0.4) == pytest.approx(0.4 * best, rel=1e-10)
