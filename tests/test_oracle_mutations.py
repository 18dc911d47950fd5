"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins catch every one: a dropped term, a wrong sign, a swapped index or a
transposed operand anywhere in the scheme must fail some pin."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ppmlr_oracle.c")

MUTANTS = {
    "slope_weight_swapped": ("(2.0 * xi[i - 1] + xi[i]) / (xi[i + 1] + xi[i])",
                             "(2.0 * xi[i + 1] + xi[i]) / (xi[i + 1] + xi[i])"),
    "edge_slope_sign": ("- x1 * z1 * dmi1 + x2 * z2 * dmi", "+ x1 * z1 * dmi1 + x2 * z2 * dmi"),
    "edge_z_swapped": ("double z1 = (x0 + x1) / (2.0 * x1 + x2);", "double z1 = (x0 + x1) / (2.0 * x2 + x1);"),
    "limiter_bound": ("double lim_m = 2.0 * fabs(dm)", "double lim_m = 4.0 * fabs(dm)"),
    "monotone_wrong_edge": ("l = 3.0 * ai - 2.0 * r;", "l = 3.0 * ai - 2.0 * l;"),
    "dod_curvature": ("(1.0 - 2.0 / 3.0 * y) * a6);\n}\ndouble orc_avg_left",
                      "(1.0 - 1.0 / 3.0 * y) * a6);\n}\ndouble orc_avg_left"),
    "riemann_pressure_sign": ("L[1] + WR * R[1] + PL - PR)", "L[1] + WR * R[1] + PR - PL)"),
    "riemann_sigma_sign": ("ZL * ZR * (vR - vL)) / (ZL + ZR);", "ZL * ZR * (vL - vR)) / (ZL + ZR);"),
    "riemann_impedance_swap": ("double Ps = (WR * PL + WL * PR", "double Ps = (WL * PL + WR * PR"),
    "lagrange_u_sign": ("double uL = b->q[1][p] - dt *", "double uL = b->q[1][p] + dt *"),
    "lagrange_energy_index": ("b->dC[6][p] = -dt * (b->rs[7][p] - b->rs[7][p - 1]);",
                              "b->dC[6][p] = -dt * (b->rs[2][p] - b->rs[2][p - 1]);"),
    "lagrange_width": ("double dxL = b->dx[p] + dt * (b->rs[0][p] - b->rs[0][p - 1]);",
                       "double dxL = b->dx[p] + dt * (b->rs[0][p + 1] - b->rs[0][p - 1]);"),
    "remap_flux_order": ("(b->dC[v][p] + b->F[v][p - 1] - b->F[v][p])", "(b->dC[v][p] + b->F[v][p] - b->F[v][p - 1])"),
    "remap_donor": ("b->F[v][p] = del * orc_avg_left(b->aL[v][p + 1], b->aR[v][p + 1], b->a6[v][p + 1], y);",
                    "b->F[v][p] = del * orc_avg_left(b->aL[v][p], b->aR[v][p], b->a6[v][p], y);"),
    "pressure_half_dropped": ("(E - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rho", "(E - (mn * mn + m1 * m1 + m2 * m2) / rho"),
    "alfven_trace_fast": ("double y = (v == 2 || v == 3) ? ya : yf;", "double y = yf;"),
    "source_curl_sign": ("double J[3] = {0.0, -DB[2], DB[1]};", "double J[3] = {0.0, DB[2], -DB[1]};"),
    "source_energy_term": ("+ BB[1][0] * cA[0] + BB[1][1] * cA[1] + BB[1][2] * cA[2];",
                           "+ BB[1][0] * cA[0] - BB[1][1] * cA[1] + BB[1][2] * cA[2];"),
    "dipole_sign": ("B[2] = M * (3.0 * mr * z + r2) / r5;", "B[2] = M * (3.0 * mr * z - r2) / r5;"),
    "outflow_ghost": ("else if (kind == BC_OUTFLOW) src = side == 0 ? 0 : N - 1;",
                      "else if (kind == BC_OUTFLOW) src = side == 0 ? 1 : N - 2;"),
    "periodic_width": ("if (c->bc[d][0] == BC_PERIODIC) lo = ((-k) % n + n) % n;",
                       "if (c->bc[d][0] == BC_PERIODIC) lo = k - 1;"),
    "source_centre_field": ("double Bd0 = b->Bd[0][p], Bd1 = b->Bd[1][p], Bd2 = b->Bd[2][p];",
                            "double Bd0 = b->Bd[0][p], Bd1 = b->Bd[2][p], Bd2 = b->Bd[1][p];"),
    "inflow_field_sign": ("double Bp[3] = {c->inflow[4] - Bdg[0]", "double Bp[3] = {c->inflow[4] + Bdg[0]"),
    "two_shock_constant": ("double a = (gamma + 1.0) / (2.0 * gamma);", "double a = (gamma - 1.0) / (2.0 * gamma);"),
    "two_shock_slope": ("double ZL = 2.0 * WLk * WLk * WLk / (WLk * WLk + CL * CL);", "double ZL = WLk;"),
    "two_shock_curve_sign": ("double uRk = R[1] + (Pc - PR) / WRk;", "double uRk = R[1] - (Pc - PR) / WRk;"),
    "two_shock_final_speed": ("WR = CR * sqrt(1.0 + a * (Pc / PR - 1.0));\n    }", "WR = CR;\n    }"),
    "steepen_one_sided_right": ("double rd = b->rq[v][p + 1] - 0.5 * b->slq[v][p + 1];",
                                "double rd = b->rq[v][p + 1] + 0.5 * b->slq[v][p + 1];"),
    "steepen_density_only": ("if (c->steepen && b->eta[p] > 0.0) {", "if (c->steepen && b->eta[p] > 0.0 && v == 0) {"),
    "steepen_curvature_test": ("if (b->d2[p + 1] * b->d2[p - 1] < 0.0 &&", "if (b->d2[p + 1] * b->d2[p - 1] > 0.0 &&"),
    "flat_omega1": ("FLAT_W1 = 0.75", "FLAT_W1 = 0.85"),
    "flat_omega2": ("FLAT_W2 = 10.0", "FLAT_W2 = 5.0"),
    "flat_epsilon": ("FLAT_EPS = 0.33", "FLAT_EPS = 0.5"),
    "flat_upwind_swapped": ("? ft[p + 1] : ft[p - 1];", "? ft[p - 1] : ft[p + 1];"),
    "flat_compression_sign": ("u[p - 1] - u[p + 1] > 0.0", "u[p + 1] - u[p - 1] > 0.0"),
    "cfl_fast_without_dipole": ("double cf = sqrt(c1 > c2 ? c1 : c2);", "double cf = sqrt(c1);"),
    "cfl_inner_not_skipped": ("if (is_inner(c, x, y, z)) continue;", "if (0 && is_inner(c, x, y, z)) continue;"),
    "cfl_no_floor": ("if (pr < c->p_min) pr = c->p_min;\n                double c1", "double c1"),
    "cfl_velocity_component": ("/ (fabs(mn / rho) + cf);", "/ (fabs(m1 / rho) + cf);"),
}

# Independent pins only: the oracle's own regression fixture
# (tests/golden/oracle_regression.json, written from the oracle) is left out,
# so each planted mistake must fail a pin fixed by the paper, a closed form, an
# exact solution or an invariant.
PINS = ["tests/test_oracle_ppm.py", "tests/test_oracle_riemann.py", "tests/test_oracle_riemann_nl.py",
        "tests/test_oracle_steepening.py",
        "tests/test_oracle_sources.py",
        "tests/test_oracle_cfl_flattening.py", "tests/test_oracle_boundaries.py",
        "tests/test_oracle_scheme.py", "tests/test_golden.py"]
DESELECT = ["tests/test_oracle_scheme.py::test_brio_wu_self_convergence",
            "tests/test_golden.py::test_oracle_regression_fixture"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, PPMLR_ORACLE_LIB=str(lib), OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *[a for d in DESELECT for a in ("--deselect", d)], *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"


# The ionosphere shell (oracle/ionosphere.py) against its own pins.
IONO_SRC = os.path.join(ROOT, "oracle", "ionosphere.py")
IONO_MUTANTS = {
    "iono_source_sign": ("rhs = (cfg.r_iono * cfg.r_iono / cfg.sigma_p) * jr[h].reshape(-1)",
                         "rhs = -(cfg.r_iono * cfg.r_iono / cfg.sigma_p) * jr[h].reshape(-1)"),
    "iono_neumann_edge": ("A[row, row] -= sp / (s * dth * dth)       # odd ghost",
                          "A[row, row] -= 0.0 * sp / (s * dth * dth)       # odd ghost"),
    "iono_pole_flux": ("sm = math.sin(th[j] - 0.5 * dth) if j > 0 else 0.0",
                       "sm = math.sin(th[j] - 0.5 * dth) if j > 0 else math.sin(0.5 * dth)"),
    "iono_phi_term": ("A[row, row] -= 2.0 / (s * s * dph * dph)", "A[row, row] -= 2.0 / (s * dph * dph)"),
    "iono_foot_exponent": ("s2i = np.where(r > 0.0, r_iono / np.where(r > 0.0, r, 1.0), np.inf) * s2",
                           "s2i = np.where(r > 0.0, (r_iono / np.where(r > 0.0, r, 1.0)) ** 1.5, np.inf) * s2"),
    "iono_hemisphere_swap": ("hemi = np.where(z >= 0.0, 0, 1)", "hemi = np.where(z >= 0.0, 1, 0)"),
    "iono_no_tube_scaling": ("jr = jpar * (bi / bm) * (br / bi)", "jr = jpar * (br / bi)"),
    "iono_radial_sign": ("jr = jpar * (bi / bm) * (br / bi)", "jr = -jpar * (bi / bm) * (br / bi)"),
    "iono_curl_component": ("return dBz_dy - dBy_dz, dBx_dz - dBz_dx, dBy_dx - dBx_dy",
                            "return dBz_dy - dBy_dz, dBz_dx - dBx_dz, dBy_dx - dBx_dy"),
    "iono_interp_transpose": ("return (1.0 - fu[idx]) * P[j, k0[idx]] + fu[idx] * P[j, k1[idx]]",
                              "return (1.0 - fu[idx]) * P[j, k1[idx]] + fu[idx] * P[j, k0[idx]]"),
    "iono_drift_sign": ("v[0, iz, iy, ix] = np.where(ok, (Ey * bz - Ez * by) / b2, 0.0)",
                        "v[0, iz, iy, ix] = np.where(ok, (Ez * by - Ey * bz) / b2, 0.0)"),
    "iono_gradient_span": ("E[d, iz, iy, ix] = -(fp - fm) / (c[hi] - c[lo])",
                           "E[d, iz, iy, ix] = -(fp - fm) / (2.0 * (c[hi] - c[lo]))"),
}


@pytest.mark.parametrize("name", sorted(IONO_MUTANTS))
def test_ionosphere_pins_catch_planted_mistake(name, tmp_path):
    old, new = IONO_MUTANTS[name]
    src = open(IONO_SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    mutated = tmp_path / "ionosphere_mut.py"
    mutated.write_text(src.replace(old, new))
    env = dict(os.environ, PPMLR_IONO_ORACLE=str(mutated))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_ionosphere.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
