"""Write tests/golden/oracle_regression.json from the oracle alone.

Regression fixture: a few seeded small runs of the oracle (one with the
ionosphere shell coupled to the inner boundary), summarised by per-variable
sums, sums of squares, sampled cells, time steps and floor counts.  Regenerate only when the oracle's arithmetic is changed on purpose,
and name in the commit message the passage (or reading) that justifies it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import ionosphere  # noqa: E402
from paper_1607_02214_gb300 import inputs  # noqa: E402

CASES = {
    "brio_wu_3d_16x6x5_5steps": lambda: (inputs.brio_wu_3d((16, 6, 5)), 5),
    "magnetosphere_24x20x20_h0_2_3steps": lambda: (
        inputs.magnetosphere(n=(24, 20, 20), h0=2.0, x_ext=(-30.0, 20.0), yz_ext=(-25.0, 25.0)), 3),
    "random_periodic_stretched_10x9x8_4steps": lambda: (inputs.Problem(
        "rand", [inputs.random_stretched_edges(k, 40 + d) for d, k in enumerate((10, 9, 8))], 5.0 / 3.0,
        inputs.BoundarySpec(powell=1), inputs.random_smooth_state((10, 9, 8), 41,
        edges=[inputs.random_stretched_edges(k, 40 + d) for d, k in enumerate((10, 9, 8))])), 4),
    "magnetosphere_28x24x24_h0_1_shell_3steps": lambda: (
        inputs.magnetosphere(n=(28, 24, 24), h0=1.0, x_ext=(-30.0, 20.0), yz_ext=(-25.0, 25.0)), 3,
        dict(r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=8, n_phi=12)),
}


def run_case(prob, nsteps, shell=None):
    bc = prob.bc
    o = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    o.set_state(prob.U0)
    dts = []
    flags = 0
    for _ in range(nsteps):
        if shell:
            v, _, _ = ionosphere.couple(o.get_state(), prob.edges, bc.dipole_moment, bc.r_inner,
                                        ionosphere.IonoConfig(**shell))
            o.set_inner_velocity(v)
        dt = o.cfl_dt(prob.cfl)
        dts.append(dt)
        flags |= o.step(dt)
    U = o.get_state()
    flat = U.reshape(8, -1)
    rng = np.random.default_rng(7)
    idx = sorted(int(i) for i in rng.choice(flat.shape[1], size=6, replace=False))
    return {"dt": dts, "flags": flags, "floors": int(o.floor_hits),
            "sum": [float(x) for x in flat.sum(axis=1)],
            "sumsq": [float(x) for x in (flat * flat).sum(axis=1)],
            "samples": {str(i): [float(x) for x in flat[:, i]] for i in idx}}


def main():
    out = {"_about": "Written by make_oracle_golden.py from the oracle only.", "cases": {}}
    for name, fn in CASES.items():
        out["cases"][name] = run_case(*fn())
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
