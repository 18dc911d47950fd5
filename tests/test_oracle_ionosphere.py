"""Pins of the oracle's ionosphere shell (Sec. II coupling; readings R1-R6 of
oracle/ionosphere.py) against closed forms:

* the cap solver converges at second order to closed-form potentials of the
  continuous equation Sigma_P Lap Phi = J_r (an m = 0 and an m = 1 mode), which
  fixes the operator, its sign, the pole and the Dirichlet edge;
* foot points are invariant along dipole field lines r = L sin^2(theta);
* a linear B' (curl constant, exact under centred differences and trilinear
  interpolation) gives the closed-form radial current on the shell, with the
  flux-tube scaling |B_d| ~ sqrt(1 + 3 cos^2) / r^3 and the dipole's radial
  direction -2 cos / sqrt(1 + 3 cos^2);
* mapped potentials are constant along field lines: the centred E on the
  inner cells is perpendicular to B_d to O(h^2), and v = E x B_d / B_d^2;
* no current, no flow: the coupled oracle step equals the plain one bit for bit.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle
from paper_1607_02214_gb300 import inputs

if os.environ.get("PPMLR_IONO_ORACLE"):          # a planted-mistake copy (tests/test_oracle_mutations.py)
    _spec = importlib.util.spec_from_file_location("iono_under_test", os.environ["PPMLR_IONO_ORACLE"])
    I = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(I)
else:
    from oracle import ionosphere as I

R_IONO, R_INNER = 1.017, 3.0


def analytic_case(m, th, ph, tmax):
    """Phi and the unit-sphere Laplacian of Phi = f(theta) cos(m phi)."""
    c = math.cos(tmax)
    if m == 0:
        f = np.cos(th) - c
        lap = -2.0 * np.cos(th)                        # (1/s)(s f')' with f' = -sin
        return f[:, None] + 0 * ph[None, :], lap[:, None] + 0 * ph[None, :]
    f = (np.cos(th) - c) * np.sin(th)
    f1 = np.cos(2 * th) - c * np.cos(th)
    f2 = -2.0 * np.sin(2 * th) + c * np.sin(th)
    lap = f2 + f1 * np.cos(th) / np.sin(th) - f / np.sin(th) ** 2
    return f[:, None] * np.cos(ph)[None, :], lap[:, None] * np.cos(ph)[None, :]


@pytest.mark.parametrize("m", [0, 1])
def test_cap_solver_converges_to_closed_form(m):
    tmax = I.cap_edge(R_IONO, R_INNER)
    errs = []
    for nt, npp in ((12, 24), (24, 48)):
        cfg = I.IonoConfig(r_iono=R_IONO, sigma_p=0.7, n_theta=nt, n_phi=npp)
        th, ph, _, _ = I.cap_grid(cfg, tmax)
        phi_a, lap = analytic_case(m, th, ph, tmax)
        jr = cfg.sigma_p * lap / R_IONO ** 2
        out = I.solve_potential(np.stack([jr, 2.0 * jr]), R_INNER, cfg)
        assert np.allclose(out[1], 2.0 * out[0], rtol=1e-12, atol=1e-14)     # linear, caps independent
        errs.append(np.max(np.abs(out[0] - phi_a)) / np.max(np.abs(phi_a)))
    assert errs[0] < 0.02, errs
    assert 3.0 < errs[0] / errs[1] < 5.0, errs                                # second order


def test_cap_grid_edge_is_foot_of_inner_equator():
    tmax = I.cap_edge(R_IONO, R_INNER)
    h, th, ph, ok = I.foot(np.array([R_INNER]), np.array([0.0]), np.array([0.0]), R_IONO)
    assert ok[0] and h[0] == 0 and abs(th[0] - tmax) < 1e-14


def test_foot_point_constant_along_field_lines():
    rng = np.random.default_rng(3)
    for L in (3.2, 5.0, 9.0):
        for phi0 in rng.uniform(0, 2 * math.pi, 3):
            for hemi, sgn in ((0, 1.0), (1, -1.0)):
                s2 = rng.uniform(R_IONO / L, 1.0, 6)             # points of the line above the shell
                th = np.arcsin(np.sqrt(s2))
                r = L * s2
                x, y, z = r * np.sin(th) * np.cos(phi0), r * np.sin(th) * np.sin(phi0), sgn * r * np.cos(th)
                h, ti, pi_, ok = I.foot(x, y, z, R_IONO)
                assert ok.all() and (h == hemi).all()
                assert np.allclose(ti, math.asin(math.sqrt(R_IONO / L)), rtol=0, atol=1e-13)
                assert np.allclose(np.cos(pi_), math.cos(phi0), atol=1e-12)
                assert np.allclose(np.sin(pi_), math.sin(phi0), atol=1e-12)
    # a line that closes inside the shell has no foot point
    h, ti, pi_, ok = I.foot(np.array([0.9]), np.array([0.0]), np.array([0.0]), R_IONO)
    assert not ok[0]


def linear_field_state(edges, a, b, c):
    cx, cy, cz = I.cell_centres(edges)
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    U = np.zeros((8,) + X.shape)
    U[0] = 1.0
    U[4], U[5], U[6] = a * Z, b * X, c * Y                   # curl = (c, a, b)
    U[7] = 1.0
    return U, (c, a, b)


def test_radial_current_of_a_linear_field():
    n = 40
    edges = [inputs.random_stretched_edges(n, 11 + d) * 14.0 - 7.0 for d in range(3)]
    a, b, c = 0.03, -0.05, 0.02
    U, J = linear_field_state(edges, a, b, c)
    M = 30.0
    cfg = I.IonoConfig(r_iono=R_IONO, r_fac=4.0, n_theta=8, n_phi=16)
    jr = I.radial_current(U, edges, M, R_INNER, cfg)
    tmax = I.cap_edge(R_IONO, R_INNER)
    th, ph, _, _ = I.cap_grid(cfg, tmax)
    for h, zs in ((0, 1.0), (1, -1.0)):
        for j, t in enumerate(th):
            s2m = cfg.r_fac / R_IONO * math.sin(t) ** 2
            if s2m > 1.0:
                assert np.all(jr[h, j] == 0.0)
                continue
            tm = math.asin(math.sqrt(s2m))
            cg_m, cg_i = zs * math.cos(tm), zs * math.cos(t)           # geographic cos(colatitude)
            for k, p in enumerate(ph):
                rp = cfg.r_fac * np.array([math.sin(tm) * math.cos(p), math.sin(tm) * math.sin(p), cg_m])
                ur = rp / cfg.r_fac
                # dipole along -z in spherical form: B = (M / r^3)(-2 cos, -sin) in (r, theta)
                uth = np.array([cg_m * math.cos(p), cg_m * math.sin(p), -math.sin(tm)])
                Bd = (M / cfg.r_fac ** 3) * (-2.0 * cg_m * ur - math.sin(tm) * uth)
                Bp = np.array([a * rp[2], b * rp[0], c * rp[1]])
                B = Bd + Bp
                jpar = np.dot(J, B) / np.linalg.norm(B)
                scale = (cfg.r_fac / R_IONO) ** 3 * math.sqrt(1 + 3 * cg_i ** 2) / math.sqrt(1 + 3 * cg_m ** 2)
                radial = -2.0 * cg_i / math.sqrt(1 + 3 * cg_i ** 2)
                assert abs(jr[h, j, k] - jpar * scale * radial) <= 1e-12 * (1 + abs(jpar * scale))


def test_mapped_potential_is_constant_along_field_lines():
    """E = -grad Phi at the inner cells is perpendicular to the dipole to
    O(h^2); v = E x B / B^2 is perpendicular to both."""
    cfg = I.IonoConfig(r_iono=R_IONO, n_theta=48, n_phi=96)
    tmax = I.cap_edge(R_IONO, R_INNER)
    th, ph, _, _ = I.cap_grid(cfg, tmax)
    phi1, _ = analytic_case(1, th, ph, tmax)
    phi = np.stack([phi1, -0.5 * phi1])
    M = 30.0
    ratios = []
    for n in (24, 48):
        e = np.linspace(-3.3, 3.3, n + 1)
        E, v = I.inner_drift(phi, [e, e, e], M, R_INNER, cfg)
        cx = I.cell_centres([e])[0]
        Z, Y, X = np.meshgrid(cx, cx, cx, indexing="ij")
        bx, by, bz = I.dipole(M, X, Y, Z)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        # cells well inside the caps' field lines, away from the pole and the edge
        s2i = R_IONO / np.maximum(r, 1e-30) * (X * X + Y * Y) / np.maximum(r * r, 1e-30)
        sel = (r < R_INNER) & (r > 1.5) & (s2i > math.sin(0.2 * tmax) ** 2) & (s2i < math.sin(0.8 * tmax) ** 2)
        Em = np.sqrt(E[0] ** 2 + E[1] ** 2 + E[2] ** 2)[sel]
        Bm = np.sqrt(bx * bx + by * by + bz * bz)[sel]
        par = np.abs(E[0] * bx + E[1] * by + E[2] * bz)[sel] / (Em * Bm)
        ratios.append(np.median(par))
        vb = np.abs(v[0] * bx + v[1] * by + v[2] * bz)[sel]
        assert np.all(vb <= 1e-12 * np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)[sel] * Bm + 1e-300)
        B2 = (bx * bx + by * by + bz * bz)[sel]
        assert np.allclose(v[0][sel], (E[1] * bz - E[2] * by)[sel] / B2, rtol=1e-12, atol=0)
    assert ratios[0] < 0.05 and ratios[1] < ratios[0] / 2.5, ratios


def test_no_current_no_flow_and_bitwise_equal_step():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    bc = pr.bc
    U = pr.U0.copy()
    U[4:7] = 0.0                                            # B' = 0: no current anywhere
    cfg = I.IonoConfig(n_theta=12, n_phi=24)
    v, phi, jr = I.couple(U, pr.edges, bc.dipole_moment, bc.r_inner, cfg)
    assert not jr.any() and not phi.any() and not v.any()

    def make():
        o = oracle.Oracle(pr.edges, pr.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                          r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
        o.set_state(U)
        return o
    a, b = make(), make()
    b.set_inner_velocity(v)
    for o in (a, b):
        for _ in range(2):
            assert o.step(o.cfl_dt(0.4)) == 0
    assert np.array_equal(a.get_state(), b.get_state())


def test_inner_flow_reaches_the_inner_cells():
    """A set flow replaces the inner state's rest flow in exactly the inner cells."""
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    bc = pr.bc
    o = oracle.Oracle(pr.edges, pr.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    o.set_state(pr.U0)
    cx, cy, cz = I.cell_centres(pr.edges)
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    inner = X * X + Y * Y + Z * Z < bc.r_inner ** 2
    v = np.zeros((3,) + X.shape)
    v[0][inner], v[1][inner], v[2][inner] = 0.01, -0.02, 0.03
    o.set_inner_velocity(v)
    assert o.step(o.cfl_dt(0.4)) == 0
    U = o.get_state()
    rho = bc.inner[0]
    assert np.allclose(U[1][inner], rho * 0.01, rtol=1e-14) and np.allclose(U[3][inner], rho * 0.03, rtol=1e-14)
    E = bc.inner[7] / (pr.gamma - 1.0) + 0.5 * rho * (0.01 ** 2 + 0.02 ** 2 + 0.03 ** 2)
    assert np.allclose(U[7][inner], E, rtol=1e-14)


def test_potential_at_nodes_pole_and_outside():
    """Points on the field line of a cap node get that node's value (either
    hemisphere); the axis gets the ring mean; lines that miss the caps get 0."""
    cfg = I.IonoConfig(r_iono=R_IONO, n_theta=10, n_phi=20)
    tmax = I.cap_edge(R_IONO, R_INNER)
    th, ph, _, _ = I.cap_grid(cfg, tmax)
    rng = np.random.default_rng(5)
    phi = rng.normal(size=(2, cfg.n_theta, cfg.n_phi))
    for h, zs in ((0, 1.0), (1, -1.0)):
        for j in (0, 3, 9):
            for k in (0, 7, 19):
                L = R_IONO / math.sin(th[j]) ** 2
                r = min(2.5, 0.9 * L)
                t = math.asin(math.sqrt(r / L))
                x = np.array([r * math.sin(t) * math.cos(ph[k])])
                y = np.array([r * math.sin(t) * math.sin(ph[k])])
                z = np.array([zs * r * math.cos(t)])
                assert abs(I.potential_at(phi, x, y, z, R_INNER, cfg)[0] - phi[h, j, k]) < 1e-9
        on_axis = I.potential_at(phi, np.array([0.0]), np.array([0.0]), np.array([zs * 2.0]), R_INNER, cfg)[0]
        assert abs(on_axis - phi[h, 0].mean()) < 1e-13
    # equatorial points inside the inner sphere: their lines close below the cap edge
    assert I.potential_at(phi, np.array([2.0]), np.array([0.5]), np.array([0.1]), R_INNER, cfg)[0] == 0.0


def test_inner_field_matches_the_gradient_of_the_mapped_potential():
    """For Phi = cos(theta) - cos(theta_max) on the caps, the mapped potential
    at (x, y, z) is sqrt(1 - s) - cos(theta_max), s = r_iono rho^2 / r^3; the
    oracle's E on the inner cells matches -grad of it to O(h^2)."""
    cfg = I.IonoConfig(r_iono=R_IONO, n_theta=64, n_phi=32)
    tmax = I.cap_edge(R_IONO, R_INNER)
    th, ph, _, _ = I.cap_grid(cfg, tmax)
    phi0, _ = analytic_case(0, th, ph, tmax)
    phi = np.stack([phi0, phi0])
    errs = []
    for n in (24, 48):
        e = np.linspace(-3.3, 3.3, n + 1)
        E, _ = I.inner_drift(phi, [e, e, e], 30.0, R_INNER, cfg)
        cx = I.cell_centres([e])[0]
        Z, Y, X = np.meshgrid(cx, cx, cx, indexing="ij")
        r = np.sqrt(X * X + Y * Y + Z * Z)
        rho2 = X * X + Y * Y
        s = R_IONO * rho2 / np.maximum(r, 1e-30) ** 3
        sel = (r < R_INNER) & (r > 1.5) & (s > math.sin(0.2 * tmax) ** 2) & (s < math.sin(0.8 * tmax) ** 2)
        r5 = np.maximum(r, 1e-30) ** 5
        ds = [R_IONO * (2 * X / r ** 3 - 3 * rho2 * X / r5), R_IONO * (2 * Y / r ** 3 - 3 * rho2 * Y / r5),
              R_IONO * (-3 * rho2 * Z / r5)]
        g = [-0.5 / np.sqrt(1 - np.clip(s, 0, 1 - 1e-12)) * d for d in ds]     # grad Phi
        num = sum((E[d] + g[d]) ** 2 for d in range(3))[sel]
        den = sum(g[d] ** 2 for d in range(3))[sel]
        errs.append(np.sqrt(np.median(num / den)))
    assert errs[0] < 0.05 and errs[1] < errs[0] / 2.5, errs
