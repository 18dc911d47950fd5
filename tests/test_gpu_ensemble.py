"""Batched ensemble and autotuners on the GPU.

Every ensemble instance must evolve like a single context advanced with
ppmlr_step_cfl from the same state (the same per-cell arithmetic and a
per-instance device dt): bit for bit on the exact FP64 path; to roundoff on
the paths compiled with contraction, whose fused multiply-adds may be formed
differently in differently inlined kernels.  Graph replay must equal direct
launches; tuned tile shapes must not change results.  FP64 instances also
match the oracle."""
import numpy as np
import pytest

from gpu_util import make_oracle, rel_l1
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def small_ensemble(seed=7):
    rng = np.random.default_rng(seed)
    shapes = [(40, 32, 32), (48, 32, 28), (36, 30, 30), (44, 34, 26), (40, 28, 36)]
    out = []
    for i, n in enumerate(shapes):
        out.append(inputs.magnetosphere(n=n, h0=1.0, n_cc=float(rng.uniform(2, 20)),
                                        vx_kms=float(rng.uniform(-800, -300)), bz_nt=float(rng.uniform(-10, 10)),
                                        name=f"m{i}"))
    return out


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_MIXED, ppmlr.PPMLR_FP64, ppmlr.PPMLR_FP64_EXACT])
def test_ensemble_equals_independent_contexts(precision):
    probs = small_ensemble()
    ens = ppmlr.Ensemble(probs, precision=precision)
    for i, p in enumerate(probs):
        ens.set_state(i, p.U0)
    nsteps = 5
    ens.step(0.4, nsteps)
    ens.check()
    dts = ens.dt()
    for i, p in enumerate(probs):
        ctx = ppmlr.Context.from_problem(p, precision)
        ctx.set_state(p.U0)
        ctx.step_cfl(0.4, nsteps)
        a, b = ens.get_state(i), ctx.get_state()
        if precision == ppmlr.PPMLR_FP64_EXACT:
            assert np.array_equal(a, b), i
            assert dts[i] == ctx.last_dt()
        else:
            tol = 1e-12 if precision == ppmlr.PPMLR_FP64 else 1e-6
            assert np.max(rel_l1(a, b)) <= tol, (i, rel_l1(a, b))
            assert abs(dts[i] - ctx.last_dt()) <= tol * dts[i]
    assert ens.diagnostics()["step"] == nsteps


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_MIXED, ppmlr.PPMLR_FP64_EXACT])
def test_ensemble_graph_equals_direct_launches_and_autotune_is_neutral(precision):
    probs = small_ensemble(11)
    a = ppmlr.Ensemble(probs, precision=precision)
    b = ppmlr.Ensemble(probs, precision=precision)
    for i, p in enumerate(probs):
        a.set_state(i, p.U0)
        b.set_state(i, p.U0)
    b.autotune()
    a.step(0.4, 4)                     # graph replay
    ms = b.time_kernels(0.4, 4)        # direct launches, tuned tiles
    assert all(v > 0 for v in ms.values())
    for i in range(len(probs)):
        if precision == ppmlr.PPMLR_FP64_EXACT:      # any launch form, bit for bit
            assert np.array_equal(a.get_state(i), b.get_state(i)), i
        else:                                        # tuned launch form may contract differently
            assert np.max(rel_l1(a.get_state(i), b.get_state(i))) <= 1e-6, i


def test_ensemble_fp64_instance_matches_oracle():
    probs = small_ensemble(3)[:2]
    ens = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_FP64)
    for i, p in enumerate(probs):
        ens.set_state(i, p.U0)
    ens.step(0.4, 3)
    for i, p in enumerate(probs):
        o = make_oracle(p)
        for _ in range(3):
            assert o.step(o.cfl_dt(0.4)) == 0
        err = rel_l1(ens.get_state(i), o.get_state())
        assert np.max(err) <= 1e-11, err


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED, ppmlr.PPMLR_FP64_EXACT])
def test_autotune_changes_speed_not_results(precision):
    p = inputs.magnetosphere(n=(56, 44, 40), h0=1.0)
    a = ppmlr.Context.from_problem(p, precision)
    b = ppmlr.Context.from_problem(p, precision)
    a.set_state(p.U0)
    b.set_state(p.U0)
    ms = b.autotune()
    assert all(m > 0 for m in ms)
    a.step_cfl(0.4, 3)
    b.step_cfl(0.4, 3)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.diagnostics()["floor_hits"] == b.diagnostics()["floor_hits"]


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
@pytest.mark.parametrize("form", [3, 5])
def test_ensemble_tma_form_matches_the_other_forms(precision, form):
    # form 3: arguments from the device table; form 5: from the kernel parameter
    probs = small_ensemble(5)
    a = ppmlr.Ensemble(probs, precision=precision)
    b = ppmlr.Ensemble(probs, precision=precision)
    b.set_launch(0, form, 124)                       # 2 pencils per x tile: divides every ny
    for axis in (1, 2):
        b.set_launch(axis, form, 256)                # TMA-staged boxes, per-instance tensor maps
    assert [t // 1000 for t in b.tiles()] == [form] * 3
    for i, p in enumerate(probs):
        a.set_state(i, p.U0)
        b.set_state(i, p.U0)
    a.step(0.4, 4)
    b.step(0.4, 4)
    b.check()
    for i in range(len(probs)):
        if precision == ppmlr.PPMLR_FP64_EXACT:
            assert np.array_equal(a.get_state(i), b.get_state(i)), i
        else:
            tol = 1e-12 if precision == ppmlr.PPMLR_FP64 else 1e-6
            assert np.max(rel_l1(b.get_state(i), a.get_state(i))) <= tol, i
    odd = ppmlr.Ensemble([inputs.magnetosphere(n=(41, 30, 30), h0=1.0)], precision=precision)
    assert odd.set_launch(1, form, 256, raise_on_error=False) == ppmlr.PPMLR_E_INVALID  # nx odd
    skew = ppmlr.Ensemble([inputs.magnetosphere(n=(40, 30, 30), h0=1.0)], precision=precision)
    assert skew.set_launch(0, form, 216, raise_on_error=False) == ppmlr.PPMLR_E_INVALID  # 4 lanes do not divide ny


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_FP64, ppmlr.PPMLR_MIXED])
def test_ensemble_persistent_parameter_form_matches_the_other_forms(precision):
    """Form 4: persistent blocks taking tiles from the work counter, every
    instance's arguments in the kernel parameter."""
    probs = small_ensemble(9)
    a = ppmlr.Ensemble(probs, precision=precision)
    b = ppmlr.Ensemble(probs, precision=precision)
    for axis in range(3):
        a.set_launch(axis, 1, 256)
        b.set_launch(axis, 4, 256)
    assert [t // 1000 for t in b.tiles()] == [4, 4, 4]
    for i, p in enumerate(probs):
        a.set_state(i, p.U0)
        b.set_state(i, p.U0)
    a.step(0.4, 4)
    b.step(0.4, 4)
    b.check()
    for i in range(len(probs)):
        if precision == ppmlr.PPMLR_FP64_EXACT:
            assert np.array_equal(a.get_state(i), b.get_state(i)), i
        else:
            tol = 1e-12 if precision == ppmlr.PPMLR_FP64 else 1e-6
            assert np.max(rel_l1(b.get_state(i), a.get_state(i))) <= tol, i
    assert a.diagnostics()["floor_hits"] == b.diagnostics()["floor_hits"]
    many = ppmlr.Ensemble([inputs.magnetosphere(n=(24, 20, 20), h0=2.0, x_ext=(-30, 20), yz_ext=(-25, 25),
                                                name=f"t{i}") for i in range(65)], precision=precision)
    for form in (2, 4, 5):                           # the kernel parameter holds at most 64 instances
        assert many.set_launch(1, form, 256, raise_on_error=False) == ppmlr.PPMLR_E_INVALID


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_MIXED])
@pytest.mark.parametrize("form", [0, 3, 4, 5])
def test_ensemble_lanes_first_tiles_match_whole_pencil_tiles(precision, form):
    """The y/z lanes-first rule (budget + 10000: chunked pencils, more lanes)
    gives the whole-pencil rule's results (bit for bit on the exact path)."""
    probs = [inputs.magnetosphere(n=n, h0=1.0, name=f"c{i}")
             for i, n in enumerate(((40, 64, 60), (36, 70, 52), (44, 50, 66)))]
    a = ppmlr.Ensemble(probs, precision=precision)
    b = ppmlr.Ensemble(probs, precision=precision)
    for axis in (1, 2):
        a.set_launch(axis, form, 256)                   # whole pencils, 2 lanes
        b.set_launch(axis, form, 10000 + 256)           # 4 lanes, pencils in chunks of 25..35 cells
    assert [t // 10000 for t in b.tiles()][1:] == [1, 1] and [t // 10000 for t in a.tiles()][1:] == [0, 0]
    assert b.set_launch(0, form, 10256, raise_on_error=False) == ppmlr.PPMLR_E_INVALID   # not along x
    for i, p in enumerate(probs):
        a.set_state(i, p.U0)
        b.set_state(i, p.U0)
    a.step(0.4, 4)
    b.step(0.4, 4)
    b.check()
    for i in range(len(probs)):
        if precision == ppmlr.PPMLR_FP64_EXACT:
            assert np.array_equal(a.get_state(i), b.get_state(i)), i
        else:
            assert np.max(rel_l1(b.get_state(i), a.get_state(i))) <= 1e-6, i
