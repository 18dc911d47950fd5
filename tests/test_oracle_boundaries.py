"""Pins of the oracle's boundary ghosts against their definitions (paper Sec.
II and Sec. IV-A boundaries; the ghost rules are the readings listed with the
design): one sweep along x of a domain with an outflow or inflow face gives
the same interior as one sweep of a wider domain whose extra cells hold, in
place of the ghosts, what the rule says the ghosts hold --

* outflow: copies of the edge cell (zero gradient), widths mirrored about
  the face;
* inflow: the fixed solar-wind state converted to conserved variables with
  B' = B_wind - B_d(cell centre), B_d the Earth dipole.

The stencil of one sweep reaches 7 zones, so the wider domain's own ghosts
(7 zones beyond the extra cells) cannot reach the compared interior.
"""
import numpy as np
import pytest

import oracle

GAM = 5.0 / 3.0
G = 7


def _dipole(M, x, y, z):
    r2 = x * x + y * y + z * z
    r5 = r2 ** 2.5
    mr = -z                                   # moment along -z
    return np.array([M * 3 * mr * x / r5, M * 3 * mr * y / r5, M * (3 * mr * z + r2) / r5])


def _cons(rho, v, Bp, p):
    v = np.asarray(v, float)
    Bp = np.asarray(Bp, float)
    return np.array([rho, *(rho * v), *Bp, p / (GAM - 1) + 0.5 * rho * v @ v + 0.5 * Bp @ Bp])


def _random_state(rng, n):
    U = np.zeros((8, 1, 1, n))
    for i in range(n):
        U[:, 0, 0, i] = _cons(rng.uniform(0.8, 1.5), rng.normal(0, 0.3, 3), rng.normal(0, 0.5, 3),
                              rng.uniform(0.5, 1.0))
    return U


def _axes(rng, n):
    ex = np.cumsum(np.r_[4.0, rng.uniform(0.5, 1.5, n)])
    return ex, np.array([-0.7, 0.6]), np.array([1.1, 1.9])


INFLOW = np.array([1.2, -0.6, 0.1, 0.05, 0.2, -0.1, 0.4, 0.7])   # rho, v, B (total), p


def _run(edges, U, bc_x, M, powell=1):
    o = oracle.Oracle(edges, GAM, [*bc_x, 1, 1, 1, 1], inflow=INFLOW, dipole_moment=M, p_min=1e-9,
                      powell=powell)
    o.set_state(U)
    flags = o.sweep(0, 0.02)
    assert flags == 0
    return o.get_state()


@pytest.mark.parametrize("M", [0.0, 30.0])
def test_outflow_ghosts_are_edge_copies(M):
    rng = np.random.default_rng(7)
    n = 12
    ex, ey, ez = _axes(rng, n)
    U = _random_state(rng, n)
    small = _run([ex, ey, ez], U, (1, 1), M)
    w = np.diff(ex)
    wl = w[:G]                                 # mirrored: the k-th ghost out has the width of cell k-1
    wr = w[::-1][:G]
    exb = np.concatenate([ex[0] - np.cumsum(wl)[::-1], ex, ex[-1] + np.cumsum(wr)])
    Ub = np.concatenate([np.repeat(U[..., :1], G, axis=-1), U, np.repeat(U[..., -1:], G, axis=-1)], axis=-1)
    big = _run([exb, ey, ez], Ub, (1, 1), M)
    np.testing.assert_allclose(small, big[..., G:G + n], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M", [0.0, 30.0])
def test_inflow_ghosts_are_the_wind_with_dipole_removed(M):
    rng = np.random.default_rng(8)
    n = 12
    ex, ey, ez = _axes(rng, n)
    U = _random_state(rng, n)
    small = _run([ex, ey, ez], U, (1, 2), M)
    w = np.diff(ex)
    wl = w[:G]
    wr = w[::-1][:G]
    right_edges = ex[-1] + np.cumsum(wr)
    exb = np.concatenate([ex[0] - np.cumsum(wl)[::-1], ex, right_edges])
    centres = 0.5 * (np.r_[ex[-1], right_edges[:-1]] + right_edges)
    yc, zc = 0.5 * (ey[0] + ey[1]), 0.5 * (ez[0] + ez[1])
    ghosts = np.zeros((8, 1, 1, G))
    for k, xc in enumerate(centres):
        Bd = _dipole(M, xc, yc, zc) if M else np.zeros(3)
        ghosts[:, 0, 0, k] = _cons(INFLOW[0], INFLOW[1:4], INFLOW[4:7] - Bd, INFLOW[7])
    Ub = np.concatenate([np.repeat(U[..., :1], G, axis=-1), U, ghosts], axis=-1)
    big = _run([exb, ey, ez], Ub, (1, 1), M)
    np.testing.assert_allclose(small, big[..., G:G + n], rtol=1e-12, atol=1e-12)
