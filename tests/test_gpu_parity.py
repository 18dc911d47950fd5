"""GPU parity: the CUDA sweeps against the FP64 oracle on the same seeded
inputs, element by element.  FP64 path: relative L1 <= 1e-11 per variable
(the stated target; both sides evaluate the same IEEE double expression trees,
so the observed difference is expected to be 0).  Mixed path: relative L1
<= 1e-5 per variable."""
import numpy as np
import pytest

from gpu_util import assert_parity, linf, make_gpu, make_oracle, rel_l1, run_pair
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_1607_02214_gb300 import build
    build.build()


def periodic_random(n, seed, stretched=True):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)] if stretched else \
        [inputs.uniform_axis(k, 0, 1) for k in n]
    U = inputs.random_smooth_state(n, seed, edges=edges)
    return inputs.Problem("rand", edges, 5.0 / 3.0, inputs.BoundarySpec(powell=1), U)


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_FP64_EXACT])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_sweep_fp64(axis, precision):
    pr = periodic_random((37, 29, 23), 3)
    o, g = make_oracle(pr), make_gpu(pr, precision)
    dt = o.cfl_dt(0.4)
    assert o.sweep(axis, dt) == 0
    g.sweep(axis, dt)
    a, b = g.get_state(), o.get_state()
    assert np.max(rel_l1(a, b)) <= FP64_TOL, rel_l1(a, b)


def test_cfl_dt_matches():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    o = make_oracle(pr)
    ref = o.cfl_dt(0.4)
    assert make_gpu(pr, ppmlr.PPMLR_FP64_EXACT).cfl_dt(0.4) == ref          # bit-identical
    assert abs(make_gpu(pr, ppmlr.PPMLR_FP64).cfl_dt(0.4) - ref) <= 1e-14 * ref
    assert abs(make_gpu(pr, ppmlr.PPMLR_MIXED).cfl_dt(0.4) - ref) <= 1e-5 * ref


@pytest.mark.parametrize("prob", ["brio_wu", "magnetosphere", "random"])
def test_exact_path_is_bit_identical(prob):
    if prob == "brio_wu":
        pr = inputs.brio_wu_3d((32, 32, 32))
    elif prob == "magnetosphere":
        pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    else:
        pr = periodic_random((37, 29, 23), 5)
    o, g, _ = run_pair(pr, 6, precision=ppmlr.PPMLR_FP64_EXACT)
    assert np.array_equal(g.get_state(), o.get_state())
    assert g.diagnostics()["floor_hits"] == o.floor_hits


def test_brio_wu_3d_32_cubed_fp64_10_steps():
    pr = inputs.brio_wu_3d((32, 32, 32))
    o, g, dts = run_pair(pr, 10)
    a, b = g.get_state(), o.get_state()
    assert np.max(rel_l1(a, b)) <= FP64_TOL, rel_l1(a, b)
    assert g.diagnostics()["floor_hits"] == o.floor_hits


def test_ragged_random_periodic_fp64():
    pr = periodic_random((37, 29, 23), 5)
    o, g, _ = run_pair(pr, 6)
    a, b = g.get_state(), o.get_state()
    assert np.max(rel_l1(a, b)) <= FP64_TOL, rel_l1(a, b)


def test_magnetosphere_small_fp64():
    pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    o, g, _ = run_pair(pr, 8)
    a, b = g.get_state(), o.get_state()
    assert np.max(rel_l1(a, b)) <= FP64_TOL, rel_l1(a, b)
    assert g.diagnostics()["floor_hits"] == o.floor_hits


def test_chunked_long_pencils_fp64():
    # pencils longer than one tile are split into chunks with 7-cell halos
    for n in ((700, 4, 3), (5, 640, 3), (3, 4, 530)):
        pr = periodic_random(n, 9)
        o, g, _ = run_pair(pr, 2)
        a, b = g.get_state(), o.get_state()
        assert np.max(rel_l1(a, b)) <= FP64_TOL, (n, rel_l1(a, b))


def test_step_cfl_matches_host_loop():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    g1 = make_gpu(pr)
    for _ in range(3):
        g1.step(g1.cfl_dt(0.4))
    g2 = make_gpu(pr)
    g2.step_cfl(0.4, 3)
    assert np.array_equal(g1.get_state(), g2.get_state())


@pytest.mark.parametrize("precision", [ppmlr.PPMLR_FP64, ppmlr.PPMLR_FP64_EXACT, ppmlr.PPMLR_MIXED])
def test_split_symmetry_gpu(precision):
    res = []
    for axis in range(3):
        pr = inputs.brio_wu_1d(40, axis=axis)
        g = make_gpu(pr, precision)
        for _ in range(8):
            g.step(g.cfl_dt(0.4))
        U = g.get_state()
        t1, t2 = (axis + 1) % 3, (axis + 2) % 3
        res.append(np.stack([U[0], U[1 + axis], U[1 + t1], U[1 + t2], U[4 + axis], U[4 + t1], U[4 + t2],
                             U[7]]).reshape(8, -1))
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_checkpoint_resume_bitwise():
    pr = inputs.magnetosphere(n=(40, 34, 30), h0=1.0)
    g = make_gpu(pr)
    for _ in range(3):
        g.step(g.cfl_dt(0.4))
    ck, step = g.get_state(), g.diagnostics()["step"]
    for _ in range(3):
        g.step(g.cfl_dt(0.4))
    ref = g.get_state()
    h = make_gpu(pr)
    h.set_state(ck)
    h.set_step_count(step)
    for _ in range(3):
        h.step(h.cfl_dt(0.4))
    assert np.array_equal(h.get_state(), ref)


def test_device_pointers_roundtrip():
    import torch
    pr = inputs.brio_wu_3d((16, 8, 8))
    g = ppmlr.Context.from_problem(pr)
    U = torch.from_numpy(pr.U0).cuda()
    g.set_state(U)
    out = torch.empty_like(U)
    g.get_state(out)
    torch.cuda.synchronize()
    assert torch.equal(out, U)


@pytest.mark.parametrize("prob", ["brio_wu", "magnetosphere"])
def test_mixed_precision(prob):
    pr = inputs.brio_wu_3d((32, 32, 32)) if prob == "brio_wu" else inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    o, g, _ = run_pair(pr, 20, precision=ppmlr.PPMLR_MIXED)
    a, b = g.get_state(), o.get_state()
    err = rel_l1(a, b)
    assert np.all(np.isfinite(a))
    assert np.max(err) <= MIXED_TOL, err


def test_high_mach_translation_fp64_exact_mixed_bounded():
    # Uniform density and velocity (100, 3, 0) with smooth pressure and field
    # perturbations: kinetic energy ~3300 x thermal energy.  The FP64 path is
    # bit-identical to the oracle.  The mixed path's FP32 remap fluxes of
    # momentum and energy carry absolute errors ~1e-7 of the kinetic energy, so
    # its recovered pressure drifts by up to ~1e-2 here: the mixed path is meant
    # for flows like the magnetosphere (kinetic/thermal ~ 50), and this bound
    # documents how far it degrades at Mach ~100.
    n = (24, 20, 18)
    edges = [inputs.uniform_axis(k, 0, 1) for k in n]
    base = inputs.random_smooth_state(n, 31, amp_v=0.0, amp_b=0.05)
    one = np.ones_like(base[0])
    p0 = 1.0 + 0.1 * np.sin(2 * np.pi * (base[0] - base[0].mean()))
    U = inputs.conserved(one, (100.0 * one, 3.0 * one, 0 * one), (base[4], base[5], base[6]), p0, 5.0 / 3.0)
    pr = inputs.Problem("mach100", edges, 5.0 / 3.0, inputs.BoundarySpec(), U)

    def pressure(X):
        return (2.0 / 3.0) * (X[7] - 0.5 * (X[1] ** 2 + X[2] ** 2 + X[3] ** 2) / X[0]
                              - 0.5 * (X[4] ** 2 + X[5] ** 2 + X[6] ** 2))
    o, g, dts = run_pair(pr, 5, precision=ppmlr.PPMLR_FP64_EXACT)
    assert np.array_equal(g.get_state(), o.get_state())
    _, gf, _ = run_pair(pr, 5, dts=dts)
    # (m_z, generated only by the field perturbations, is a weak component here)
    assert_parity(gf.get_state(), o.get_state(), FP64_TOL, 1e-9)
    _, gm, _ = run_pair(pr, 5, precision=ppmlr.PPMLR_MIXED, dts=dts)
    pa, pb = pressure(gm.get_state()), pressure(o.get_state())
    assert np.all(pb > 0.5)
    rel = np.abs(pa - pb) / pb
    assert rel.max() < 5e-2 and rel.mean() < 5e-3, (rel.max(), rel.mean())
