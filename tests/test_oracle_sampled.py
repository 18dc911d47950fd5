"""The oracle's sampled-pencil sweep equals the same pencils of a full sweep
(it is used for parity checks on grids too large to sweep whole)."""
import numpy as np

import oracle
from paper_1607_02214_gb300 import inputs


def test_sampled_sweep_matches_full_sweep():
    pr = inputs.magnetosphere(n=(40, 32, 30), h0=1.0)
    bc = pr.bc
    mk = lambda: oracle.Oracle(pr.edges, pr.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                               r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    rng = np.random.default_rng(1)
    for axis in range(3):
        o = mk()
        o.set_state(pr.U0)
        dt = o.cfl_dt(0.4)
        a1, a2 = [d for d in range(3) if d != axis]
        j = rng.integers(0, pr.n[a1], size=7)
        k = rng.integers(0, pr.n[a2], size=7)
        got, fl = o.sweep_sampled(axis, dt, j, k)
        assert fl == 0
        assert np.array_equal(o.get_state(), pr.U0)          # state untouched
        o.sweep(axis, dt)
        U = o.get_state()
        for q in range(len(j)):
            idx = [slice(None)] * 3                            # (z, y, x)
            idx[2 - axis] = slice(None)
            idx[2 - a1] = j[q]
            idx[2 - a2] = k[q]
            ref = U[(slice(None),) + tuple(idx)]
            assert np.array_equal(got[q], ref)
