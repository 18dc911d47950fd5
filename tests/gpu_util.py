"""Helpers shared by the GPU tests: run the GPU library and the oracle on the
same seeded inputs and compare."""
import numpy as np

import oracle
from paper_1607_02214_gb300 import inputs, ppmlr


def make_oracle(prob):
    bc = prob.bc
    o = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    o.set_state(prob.U0)
    return o


def make_gpu(prob, precision=ppmlr.PPMLR_FP64):
    c = ppmlr.Context.from_problem(prob, precision)
    c.set_state(prob.U0)
    return c


def group_scales(U):
    """L1 scale per variable: its own group's sum (rho; momentum; B'; E)."""
    a = np.abs(U).reshape(8, -1).sum(axis=1)
    m, b = a[1:4].sum(), a[4:7].sum()
    return np.array([a[0], m, m, m, b, b, b, a[7]])


def rel_l1(a, b):
    """Per-variable relative L1 of a against reference b, the definition:
    sum|a - b| / sum|b| over the cells, for each of the 8 variables.  A
    variable whose reference is zero to roundoff (sum|b| below 1e-12 of its
    group's sum -- rho; momentum; B'; E), such as m_y of a shock tube along x,
    is scaled by its group's sum instead."""
    d = np.abs(a - b).reshape(8, -1).sum(axis=1)
    own = np.abs(b).reshape(8, -1).sum(axis=1)
    grp = group_scales(b)
    s = np.where(own > 1e-12 * grp, own, grp)
    return d / np.maximum(s, 1e-300 * a[0].size)


def rel_l1_group(a, b):
    """Per-variable L1 of a against b, each scaled by its group's reference sum."""
    d = np.abs(a - b).reshape(8, -1).sum(axis=1)
    return d / np.maximum(group_scales(b), 1e-300 * a[0].size)


def linf(a, b):
    return np.abs(a - b).reshape(8, -1).max(axis=1)


def run_pair(prob, nsteps, precision=ppmlr.PPMLR_FP64, dts=None):
    """Advance oracle and GPU with the oracle's CFL time steps (or given dts)."""
    o = make_oracle(prob)
    g = make_gpu(prob, precision)
    used = []
    for k in range(nsteps):
        dt = dts[k] if dts is not None else o.cfl_dt(prob.cfl)
        used.append(dt)
        assert o.step(dt) == 0
        g.step(dt)
    return o, g, used


def weak_components(b, frac=1e-2):
    """Variables whose reference sum is below `frac` of their group's sum
    (e.g. the transverse momenta of a flow along x)."""
    own = np.abs(b).reshape(8, -1).sum(axis=1)
    return own < frac * group_scales(b)


def assert_parity(a, b, tol, weak_tol):
    """The strict per-variable relative L1 of a against b within `tol` for
    every variable, except the weak components (reference sum below 1% of the
    group's), whose strict figure is held to `weak_tol`; every variable's
    group-scaled figure within `tol`.  Returns (strict, group-scaled)."""
    err, errg = rel_l1(a, b), rel_l1_group(a, b)
    weak = weak_components(b)
    assert np.all(err[~weak] <= tol), (err, weak)
    assert np.all(err[weak] <= weak_tol), (err, weak)
    assert np.all(errg <= tol), errg
    return err, errg
