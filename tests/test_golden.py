"""Golden fixtures: the paper's stated constants, and the oracle's regression
fixture (written by tests/golden/make_oracle_golden.py from the oracle only)."""
import json
import math
import os

import numpy as np
import pytest

from paper_1607_02214_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_paper_constants_used_by_the_workloads():
    c = load("paper_constants.json")
    assert inputs.magnetosphere(n=(24, 20, 20), h0=2.0, x_ext=(-30, 20), yz_ext=(-25, 25)).gamma == c["gamma"]["value"]
    assert math.isclose(inputs.MU0, c["mu0_si"]["value"], rel_tol=1e-15)
    pr = inputs.magnetosphere(n=(24, 20, 20), h0=2.0, x_ext=(-30, 20), yz_ext=(-25, 25))
    assert pr.bc.r_inner == c["inner_boundary_re"]["value"]


def test_paper_grid_stretch_ratio():
    # The paper's y/z axes (150 cells over +-100 R_E, 0.4 R_E core within
    # 10 R_E) imply the 1.05 stretch ratio it states.
    c = load("paper_constants.json")
    g, s = c["grid"], c["stretch"]
    e, (rl, rh) = inputs.stretched_axis(g["n"][1], g["yz"][0], g["yz"][1], g["h0"], core=s["core_re"])
    assert abs(rl - s["ratio"]) < 2e-3 and abs(rh - s["ratio"]) < 2e-3
    assert abs(np.diff(e).min() - g["h0"]) < 1e-12


def test_initial_state_image_dipole_split():
    # B = B_d + B' has no x component on the plane x = 15 R_E on the image side.
    c = load("paper_constants.json")["initial_state"]
    M = inputs.dipole_moment_code()
    y, z = np.array([3.0, -7.0, 0.5]), np.array([4.0, 2.5, -9.0])
    x0 = c["split_x"]
    bdx = inputs.dipole_field(M, x0, y, z)[0]
    bix = inputs.dipole_field(M, x0 - c["image_dipole_at"][0], y, z)[0]
    assert np.max(np.abs(bdx + bix)) < 1e-12 * M


def test_oracle_regression_fixture():
    import oracle
    from golden.make_oracle_golden import CASES, run_case
    gold = load("oracle_regression.json")["cases"]
    for name, fn in CASES.items():
        got = run_case(*fn())
        ref = gold[name]
        assert got["flags"] == ref["flags"] and got["floors"] == ref["floors"]
        np.testing.assert_allclose(got["dt"], ref["dt"], rtol=1e-13)
        np.testing.assert_allclose(got["sum"], ref["sum"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got["sumsq"], ref["sumsq"], rtol=1e-12)
        for k, v in ref["samples"].items():
            np.testing.assert_allclose(got["samples"][k], v, rtol=1e-12, atol=1e-13)
