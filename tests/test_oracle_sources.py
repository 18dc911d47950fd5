"""Pins for the dipole-coupling and Powell source terms of the MHD system in
B' form (Sec. II):
    d(rho v)/dt  += (curl B') x B_d
    dB'/dt       += curl(v x B_d) - v div B'
    dE/dt        += v . [(curl B') x B_d] + B' . curl(v x B_d)
The oracle applies them split by direction inside each sweep.  Switching the
dipole (or the Powell term) on and off on the same state isolates them: over
one step with a tiny dt the difference must equal dt times the right-hand side
above, evaluated here in vector form with central differences."""
import numpy as np
import pytest

import oracle
from paper_1607_02214_gb300 import inputs


def grad(f, h, axis):
    # array axes are (z, y, x); spatial axis 0 = x -> array axis 2
    ax = 2 - axis
    return (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / (2 * h)


def curl(F, h):
    Fx, Fy, Fz = F
    return np.stack([grad(Fz, h, 1) - grad(Fy, h, 2),
                     grad(Fx, h, 2) - grad(Fz, h, 0),
                     grad(Fy, h, 0) - grad(Fx, h, 1)])


def one_step_delta(U, edges, M, powell, dt):
    o = oracle.Oracle(edges, 5 / 3, [0] * 6, dipole_moment=M, powell=powell, p_min=1e-12)
    o.set_state(U)
    assert o.step(dt) == 0
    return o.get_state() - U


def test_dipole_and_powell_sources_match_pde():
    n = 16
    lo, hi = 4.0, 10.0                       # a box away from the dipole's centre
    h = (hi - lo) / n
    edges = [inputs.uniform_axis(n, lo, hi) for _ in range(3)]
    U = inputs.random_smooth_state((n, n, n), 21, edges=[inputs.uniform_axis(n, 0, 1)] * 3)
    M = 50.0
    dt = 1e-7
    dM = one_step_delta(U, edges, M, 0, dt) - one_step_delta(U, edges, 0.0, 0, dt)
    dP = one_step_delta(U, edges, 0.0, 1, dt) - one_step_delta(U, edges, 0.0, 0, dt)

    xc = inputs.centres(edges[0])
    x, y, z = np.broadcast_arrays(xc[None, None, :], xc[None, :, None], xc[:, None, None])
    Bd = np.stack(inputs.dipole_field(M, x, y, z))
    rho = U[0]
    v = U[1:4] / rho
    Bp = U[4:7]
    J = curl(Bp, h)
    Sm = np.cross(J, Bd, axis=0)
    cA = curl(np.cross(v, Bd, axis=0), h)
    SE = (v * Sm).sum(0) + (Bp * cA).sum(0)
    divB = grad(Bp[0], h, 0) + grad(Bp[1], h, 1) + grad(Bp[2], h, 2)

    inner = (slice(1, -1),) * 3             # central differences need both neighbours
    def check(got, ref):
        got, ref = got[inner], ref[inner]
        scale = np.max(np.abs(ref))
        assert scale > 0
        assert np.max(np.abs(got - ref)) < 1e-4 * scale, np.max(np.abs(got - ref)) / scale

    for k in range(3):
        check(dM[1 + k] / dt, Sm[k])
        check(dM[4 + k] / dt, cA[k])
        check(dP[4 + k] / dt, -v[k] * divB)
    check(dM[7] / dt, SE)
    # no mass source: density differs only by roundoff of the later sweeps
    assert np.max(np.abs(dM[0])) < 1e-13 and np.max(np.abs(dP[0])) < 1e-13
    # the Powell term acts on B' only (other components: roundoff)
    assert np.max(np.abs(dP[[1, 2, 3, 7]])) < 1e-13
