"""Launch forms of the y and z sweeps with TMA-staged input boxes (persistent
double-buffered, and one tile per block) give the same results as the
one-block-per-tile form that reads global memory: bit for bit on the exact
FP64 path, to roundoff on the contracted paths.  Includes periodic axes whose
ghosts wrap inside the box, chunked pencils whose ghosts come from outside it,
ragged lane groups and inflow/outflow/inner-sphere boundaries."""
import numpy as np
import pytest

from gpu_util import make_gpu, rel_l1
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def periodic_random(n, seed):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    return inputs.Problem("rand", edges, 5.0 / 3.0, inputs.BoundarySpec(powell=1),
                          inputs.random_smooth_state(n, seed, edges=edges))


CASES = {
    "magnetosphere": lambda: inputs.magnetosphere(n=(48, 40, 36), h0=1.0),
    "periodic_ragged": lambda: periodic_random((38, 29, 23), 4),
    "chunked": lambda: periodic_random((6, 300, 290), 8),
}
# forced (axis, C, L).  x: C even and L dividing ny (the x-sweep box holds L
# pencils of one z plane); chunked y/z: three chunks per pencil, the last ragged
TILES = {"magnetosphere": [(0, 48, 4)], "periodic_ragged": [(0, 38, 1)],
         "chunked": [(0, 6, 4), (1, 100, 2), (2, 97, 2)]}


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("form", [1, 2])
def test_tma_forms_match_plain(case, precision, form):
    pr = CASES[case]()
    ref = make_gpu(pr, precision)
    got = make_gpu(pr, precision)
    for axis, C, L in TILES.get(case, []):
        ref.set_tiles(axis, C, L)
        got.set_tiles(axis, C, L)
        assert got.tiles()[0][axis] == C and got.tiles()[1][axis] == L
    used, why = 0, []
    for axis in (0, 1, 2):
        if got.set_sweep_form(axis, form, raise_on_error=False) == ppmlr.PPMLR_OK:
            used += 1
        else:
            why.append(ppmlr.load().ppmlr_last_error(got._h).decode())
    assert used >= (3 if form == 2 else 2), why       # x has the one-tile form only
    assert got.sweep_forms()[1:] == [form, form]
    assert got.sweep_forms()[0] == (form if form == 2 else 0)
    for _ in range(3):
        dt = ref.cfl_dt(0.4)
        ref.step(dt)
        got.step(dt)
    got.check()
    a, b = got.get_state(), ref.get_state()
    if precision == ppmlr.PPMLR_FP64_EXACT:
        assert np.array_equal(a, b)
    else:
        tol = 1e-12 if precision == ppmlr.PPMLR_FP64 else 1e-6
        assert np.max(rel_l1(a, b)) <= tol, rel_l1(a, b)


def test_set_tiles_bounds():
    got = make_gpu(CASES["periodic_ragged"](), ppmlr.PPMLR_FP64)
    before = got.tiles()
    for axis, C, L in [(3, 10, 1), (-1, 10, 1), (1, 0, 1), (1, 30, 1), (1, 10, 0), (0, 38, 12), (1, 15, 16)]:
        with pytest.raises(ppmlr.PPMLRError):
            got.set_tiles(axis, C, L)
    assert got.tiles() == before
    got.set_sweep_form(2, 2)
    got.set_tiles(2, 23, 4)
    assert got.sweep_forms()[2] == 0


def test_fp64_x_tiles_above_the_general_budget():
    # the contracted FP64 x sweep takes tiles of up to 576 threads (its
    # kernel's register cap leaves room for them); the other forms and
    # directions keep their budgets
    pr = CASES["magnetosphere"]()
    ref = make_gpu(pr, ppmlr.PPMLR_FP64)
    got = make_gpu(pr, ppmlr.PPMLR_FP64)
    got.set_tiles(0, 48, 8)                       # 62 x 8 = 496 threads
    assert got.tiles()[0][0] == 48 and got.tiles()[1][0] == 8
    with pytest.raises(ppmlr.PPMLRError):
        got.set_tiles(1, 40, 16)                  # 54 x 16 = 864
    with pytest.raises(ppmlr.PPMLRError):
        make_gpu(pr, ppmlr.PPMLR_FP64_EXACT).set_tiles(0, 48, 8)
    for _ in range(3):
        dt = ref.cfl_dt(0.4)
        ref.step(dt)
        got.step(dt)
    got.check()
    assert np.max(rel_l1(got.get_state(), ref.get_state())) <= 1e-12
