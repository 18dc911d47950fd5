"""Contact steepening on the GPU against the oracle's: bit for bit on the exact
FP64 path (single pencils, chunked pencils, every sweep direction, TMA-staged
and global-memory forms, the ensemble), to the FP64 and mixed tolerances on
the other paths."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle, rel_l1
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

G53 = 5.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def contact(axis):
    return inputs.shock_tube_1d(160, (1.0, 1.0, 0.2, 0, 0.3, 0.5, 0, 1.0), (0.125, 1.0, 0.2, 0, 0.3, 0.5, 0, 1.0),
                                G53, axis=axis, periodic=True)


def periodic_random(n, seed):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    return inputs.Problem("rand", edges, G53, inputs.BoundarySpec(powell=1),
                          inputs.random_smooth_state(n, seed, edges=edges))


CASES = {
    "contact_x": lambda: contact(0),
    "contact_y": lambda: contact(1),
    "contact_z": lambda: contact(2),
    "brio_wu": lambda: inputs.brio_wu_3d((32, 32, 32)),
    "magnetosphere": lambda: inputs.magnetosphere(n=(48, 40, 36), h0=1.0),
}


def pair(pr, precision, nsteps, tiles=(), forms=()):
    o = make_oracle(pr)
    o.set_steepening(1)
    g = make_gpu(pr, precision)
    g.set_steepening(1)
    for axis, C, L in tiles:
        g.set_tiles(axis, C, L)
    for axis, f in forms:
        g.set_sweep_form(axis, f)
    for _ in range(nsteps):
        dt = o.cfl_dt(pr.cfl)
        assert o.step(dt) == 0
        g.step(dt)
    return o, g


@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_path_is_bit_identical(case):
    o, g = pair(CASES[case](), ppmlr.PPMLR_FP64_EXACT, 6)
    assert np.array_equal(g.get_state(), o.get_state())


def test_exact_path_chunked_and_tma_staged():
    pr = periodic_random((6, 300, 290), 8)
    o, g = pair(pr, ppmlr.PPMLR_FP64_EXACT, 3, tiles=[(0, 6, 4), (1, 100, 2), (2, 97, 2)],
                forms=[(0, 2), (1, 2), (2, 2)])
    assert g.sweep_forms() == [2, 2, 2]
    assert np.array_equal(g.get_state(), o.get_state())


@pytest.mark.parametrize("case", ["contact_x", "brio_wu", "magnetosphere"])
@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
def test_contracted_paths_within_tolerance(case, precision):
    o, g = pair(CASES[case](), precision, 10)
    err = rel_l1(g.get_state(), o.get_state())
    assert np.max(err) <= (1e-11 if precision == ppmlr.PPMLR_FP64 else 1e-5), err


def test_steepening_sharpens_the_contact_on_the_gpu():
    pr = contact(0)
    a, b = make_gpu(pr), make_gpu(pr)
    b.set_steepening(1)
    for g in (a, b):
        g.run(pr.cfl, 200, graph_steps=8)
    rho_a, rho_b = a.get_state()[0].ravel(), b.get_state()[0].ravel()
    width = lambda r: int(((r > 0.2125) & (r < 0.9125)).sum())
    assert width(rho_b) < width(rho_a)


def test_ensemble_instances_match_the_oracle():
    from test_gpu_ensemble import small_ensemble
    probs = small_ensemble(9)[:3]
    ens = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_FP64_EXACT)
    ens.set_steepening(1)
    for i, p in enumerate(probs):
        ens.set_state(i, p.U0)
    ens.step(0.4, 3)
    for i, p in enumerate(probs):
        o = make_oracle(p)
        o.set_steepening(1)
        for _ in range(3):
            assert o.step(o.cfl_dt(0.4)) == 0
        assert np.array_equal(ens.get_state(i), o.get_state()), i
