"""Cases run against the bounds-checked build of the library (set
PPMLR_LIBRARY to it): every status must be OK -- no kernel index left its
array -- and the exact path must still match the oracle bit for bit.  Run as a
script by test_gpu_checked.py; exits non-zero on the first failure."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from gpu_util import make_gpu, make_oracle  # noqa: E402
from paper_1607_02214_gb300 import inputs, ppmlr  # noqa: E402


def periodic_random(n, seed):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    return inputs.Problem("rand", edges, 5.0 / 3.0, inputs.BoundarySpec(powell=1),
                          inputs.random_smooth_state(n, seed, edges=edges))


def against_oracle(pr, nsteps, tiles=(), forms=(), riemann=0, steepen=0):
    o = make_oracle(pr)
    o.set_riemann(riemann)
    o.set_steepening(steepen)
    g = make_gpu(pr, ppmlr.PPMLR_FP64_EXACT)
    g.set_riemann_solver(riemann)
    g.set_steepening(steepen)
    for axis, C, L in tiles:
        g.set_tiles(axis, C, L)
    for axis, f in forms:
        g.set_sweep_form(axis, f)
    for _ in range(nsteps):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    g.check()                                     # raises PPMLRError on PPMLR_E_BOUNDS
    assert np.array_equal(g.get_state(), o.get_state())


def main():
    assert os.environ.get("PPMLR_LIBRARY", "").endswith("_check.so"), "run with the checked library"
    mag = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    against_oracle(mag, 3, tiles=[(0, 48, 4)], forms=[(0, 2), (1, 2), (2, 2)], riemann=4, steepen=1)
    against_oracle(mag, 3, forms=[(1, 1), (2, 1)])
    against_oracle(periodic_random((38, 29, 23), 4), 3, steepen=1)
    against_oracle(periodic_random((6, 300, 290), 8), 2, tiles=[(0, 6, 4), (1, 100, 2), (2, 97, 2)],
                   forms=[(0, 2), (1, 2), (2, 2)])
    for precision in (ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED):
        g = make_gpu(mag, precision)
        g.autotune()
        g.set_steepening(1)
        g.run(mag.cfl, 4, graph_steps=2)
        g.check()
    from test_gpu_ensemble import small_ensemble
    probs = small_ensemble(5)
    for precision in (ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_MIXED):
        ens = ppmlr.Ensemble(probs, precision=precision)
        ens.set_launch(0, 3, 124)
        ens.set_launch(1, 3, 256)
        ens.set_launch(2, 2, 256)
        ens.set_steepening(1)
        for i, p in enumerate(probs):
            ens.set_state(i, p.U0)
        ens.step(0.4, 2)
        ens.check()
    print("checked build: all cases OK")


if __name__ == "__main__":
    main()
