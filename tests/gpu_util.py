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
    """Per-variable relative L1 of a against reference b."""
    d = np.abs(a - b).reshape(8, -1).sum(axis=1)
    s = np.maximum(group_scales(b), 1e-300 * a[0].size)
    return d / s


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
