"""Whole-scheme pins for the oracle: exact Sod solution, Brio-Wu
self-convergence, linear Alfven-wave order, conservation, equilibria,
dimensional-split symmetry, thread-count independence and a magnetosphere
smoke run."""
import numpy as np
import pytest

import oracle
from exact_riemann import sample
from paper_1607_02214_gb300 import inputs


def make(prob, **kw):
    bc = prob.bc
    o = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell, **kw)
    o.set_state(prob.U0)
    return o


def test_sod_converges_to_exact_solution():
    errs = []
    for n in (100, 200, 400, 800):
        pr = inputs.sod(n)
        o = make(pr)
        t, k, flags = o.run(0.4, t_end=0.2)
        assert flags == 0 and o.floor_hits == 0
        U = o.get_state()[:, 0, 0, :]
        xc = inputs.centres(pr.edges[0])
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, (xc - 0.5) / 0.2)
        errs.append(np.mean(np.abs(U[0] - ex[0])))
        # mass and energy are conserved while no wave reaches the outflow ends
        assert abs(U[0].mean() - 0.5625) < 1e-14
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert errs[0] < 8e-3                      # PPM-quality profile at N = 100
    assert np.all(orders > 0.8)                # first order at discontinuities


def test_brio_wu_self_convergence():
    def run(n):
        pr = inputs.brio_wu_1d(n)
        o = make(pr)
        _, _, flags = o.run(0.4, t_end=0.1)
        assert flags == 0
        return o.get_state()[:, 0, 0, :]
    ref_n = 2048
    ref = run(ref_n)
    errs = []
    for n in (64, 128, 256):
        U = run(n)
        r = ref.reshape(8, n, ref_n // n).mean(axis=2)
        errs.append(np.mean(np.abs(U[0] - r[0])) + np.mean(np.abs(U[5] - r[5])))
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0)
    assert np.all(np.log2(errs[:-1] / errs[1:]) > 0.5)


def test_alfven_wave_order():
    errs = []
    for n in (32, 64, 128, 256):
        pr = inputs.alfven_wave_1d(n)
        o = make(pr)
        _, _, flags = o.run(0.4, t_end=1.0)   # one period at v_A = 1
        assert flags == 0
        U = o.get_state()
        errs.append(np.mean(np.abs(U[5] - pr.U0[5])))
    errs = np.array(errs)
    order = np.log2(errs[0] / errs[-1]) / 3.0
    assert order > 1.5, (errs, order)


def periodic_random(n, seed, stretched=False):
    edges = None
    if stretched:
        edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    U = inputs.random_smooth_state(n, seed, edges=edges)
    if edges is None:
        edges = [inputs.uniform_axis(k, 0, 1) for k in n]
    return inputs.Problem("rand", edges, 5.0 / 3.0, inputs.BoundarySpec(), U)


@pytest.mark.parametrize("stretched", [False, True])
def test_conservation_periodic(stretched):
    pr = periodic_random((12, 10, 9), 5, stretched)
    o = make(pr)
    V = (np.diff(pr.edges[2])[:, None, None] * np.diff(pr.edges[1])[None, :, None]
         * np.diff(pr.edges[0])[None, None, :])
    tot0 = np.array([(pr.U0[v] * V).sum() for v in range(8)])
    scale = np.array([(np.abs(pr.U0[v]) * V).sum() for v in range(8)])
    _, k, flags = o.run(0.4, nsteps=30)
    assert flags == 0
    U = o.get_state()
    tot = np.array([(U[v] * V).sum() for v in range(8)])
    assert np.max(np.abs(tot - tot0) / scale) < 1e-13
    assert not np.allclose(U, pr.U0)


def test_uniform_state_is_exact():
    n = (9, 8, 7)
    edges = [inputs.random_stretched_edges(n[d], 11 + d) for d in range(3)]
    one = np.ones((n[2], n[1], n[0]))
    U = inputs.conserved(1.3 * one, (0.4 * one, -0.7 * one, 0.2 * one), (0.5 * one, 0.1 * one, -0.8 * one),
                         0.9 * one, 5 / 3)
    pr = inputs.Problem("uni", edges, 5 / 3, inputs.BoundarySpec(face=((1, 1), (0, 0), (1, 1))), U)
    o = make(pr)
    o.run(0.4, nsteps=5)
    assert np.array_equal(o.get_state(), U)


def test_dipole_equilibrium_is_exact():
    pr = inputs.magnetosphere(n=(24, 20, 20), h0=2.0, x_ext=(-30, 20), yz_ext=(-25, 25))
    # plasma at rest, B' = 0, uniform rho and p, dipole and inner sphere on, outflow faces
    rho, p = 5.0, 0.8
    nz, ny, nx = pr.U0.shape[1:]
    one = np.ones((nz, ny, nx))
    z = 0 * one
    U = inputs.conserved(rho * one, (z, z, z), (z, z, z), p * one, pr.gamma)
    bc = pr.bc
    bc.face = ((1, 1), (1, 1), (1, 1))
    bc.inner = (rho, 0, 0, 0, 0, 0, 0, p)
    pr.U0 = U
    o = make(pr)
    _, _, flags = o.run(0.4, nsteps=4)
    assert flags == 0
    assert np.array_equal(o.get_state(), U)


def test_split_symmetry_is_bitwise():
    # A 1D problem along x, y or z (states given in the sweep's local frame)
    # gives identical results.
    res = []
    for axis in range(3):
        pr = inputs.brio_wu_1d(48, axis=axis)
        o = make(pr)
        o.run(0.4, nsteps=12)
        U = o.get_state()
        t1, t2 = (axis + 1) % 3, (axis + 2) % 3
        loc = np.stack([U[0], U[1 + axis], U[1 + t1], U[1 + t2], U[4 + axis], U[4 + t1], U[4 + t2], U[7]])
        res.append(loc.reshape(8, -1))
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_replicated_columns_identical_and_thread_independent():
    pr = inputs.brio_wu_3d((24, 6, 5))
    outs = []
    for threads in (1, 3):
        oracle.set_threads(threads)
        o = make(pr)
        o.run(0.4, nsteps=6)
        outs.append(o.get_state())
    oracle.set_threads(0)
    assert np.array_equal(outs[0], outs[1])
    U = outs[0]
    assert np.array_equal(U, np.broadcast_to(U[:, :1, :1, :], U.shape))


def test_inflow_keeps_matching_uniform_wind():
    # Uniform wind with no dipole, inflow state equal to the wind: unchanged.
    pr = inputs.magnetosphere(n=(20, 16, 16), h0=2.0, x_ext=(-40, 30), yz_ext=(-30, 30))
    pr.bc.dipole_moment = 0.0
    pr.bc.r_inner = 0.0
    rho, vx, _, _, _, _, bz, p = pr.bc.inflow
    nz, ny, nx = pr.U0.shape[1:]
    one = np.ones((nz, ny, nx))
    U = inputs.conserved(rho * one, (vx * one, 0 * one, 0 * one), (0 * one, 0 * one, bz * one), p * one, pr.gamma)
    pr.U0 = U
    o = make(pr)
    o.run(0.4, nsteps=3)
    assert np.array_equal(o.get_state(), U)


def test_magnetosphere_smoke():
    pr = inputs.magnetosphere(n=(40, 32, 32), h0=1.0)
    o = make(pr)
    dts = []
    for _ in range(10):
        dt = o.cfl_dt(pr.cfl)
        assert np.isfinite(dt) and dt > 0
        dts.append(dt)
        assert o.step(dt) == 0
    U = o.get_state()
    assert np.all(np.isfinite(U))
    assert np.all(U[0] > 0)
    # the inner sphere holds its fixed state
    x = inputs.centres(pr.edges[0])[None, None, :]
    y = inputs.centres(pr.edges[1])[None, :, None]
    z = inputs.centres(pr.edges[2])[:, None, None]
    inside = np.broadcast_to(x * x + y * y + z * z < 9.0, U.shape[1:])
    assert inside.any()
    assert np.all(U[1:7][:, inside] == 0.0)


def test_stretched_grid_generator():
    for n, lo, hi, h0 in ((256, -100, 30, 0.4), (192, -60, 60, 0.4), (96, -60, 60, 0.4), (512, -100, 30, 0.2)):
        e, (rl, rh) = inputs.stretched_axis(n, lo, hi, h0)
        w = np.diff(e)
        assert len(e) == n + 1 and e[0] == lo and e[-1] == hi
        assert np.all(w > 0)
        assert abs(w.min() - h0) < 1e-9
        core = (e[:-1] >= -10 - 1e-9) & (e[1:] <= 10 + 1e-9)
        assert np.allclose(w[core], h0)
        i0 = np.argmin(np.abs(e + 10))
        assert np.all(np.diff(w[:i0][::-1]) > 0)       # grows outward on the low side
        assert rl > 1 and rh > 1
    # the magnetosphere y/z axes of 192 cells stretch by about 1.015
    _, (rl, rh) = inputs.stretched_axis(192, -60, 60, 0.4)
    assert abs(rl - 1.015) < 0.003 and abs(rh - 1.015) < 0.003
