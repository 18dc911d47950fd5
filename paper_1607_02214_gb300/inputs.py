"""Seeded synthetic workloads: grids, initial states and boundary specifications.

This module builds INPUTS only.  It holds none of the sweep's arithmetic and is
the one module that both the GPU library's callers and the CPU reference
consume.  The closure E = p/(gamma-1) + rho v^2/2 + |B'|^2/2 and the dipole
formula appear here only to define initial data.

Workloads (the paper's runs use a 156x150x150 stretched magnetosphere grid
that is not available as data; these synthetic inputs stand in for it):

* ``brio_wu_3d``      -- uniform periodic cube, Brio-Wu states along x,
                         replicated in y and z (gamma = 5/3).
* ``magnetosphere``   -- stretched Cartesian grid (uniform core of width h0
                         within 10 R_E, geometric stretch outward, Sec. III-B),
                         Earth dipole, inner sphere r = 3 R_E, solar-wind inflow
                         at x = +30 R_E and outflow elsewhere; initial state of
                         Sec. IV-A (image dipole for x <= 15 R_E, uniform solar
                         wind and IMF beyond).
* ``ensemble``        -- 48 magnetosphere instances on uneven grids with seeded
                         solar-wind inputs.
* 1D problems (Sod, Brio-Wu, Alfven wave) and random smooth periodic states for
  the tests.

Units: length R_E = 6371.2 km, velocity v0 = 100 km/s, number density
n0 = 1 cm^-3 (rho0 = m_p n0), field sqrt(mu0 rho0) v0 = 4.585 nT, pressure
rho0 v0^2 = 1.6726e-11 Pa, time R_E / v0 = 63.7 s; mu0 = 1 in code units.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

# ---- physical units ---------------------------------------------------------
MU0 = 4e-7 * math.pi
M_P = 1.67262192e-27
K_B = 1.380649e-23
R_E_KM = 6371.2
V0 = 1.0e5                      # m/s
N0 = 1.0e6                      # m^-3
RHO0 = M_P * N0
B_UNIT_NT = math.sqrt(MU0 * RHO0) * V0 * 1e9
P_UNIT = RHO0 * V0 * V0
B_EARTH_NT = 3.0e4              # equatorial surface field

BC_PERIODIC, BC_OUTFLOW, BC_INFLOW = 0, 1, 2


@dataclasses.dataclass
class BoundarySpec:
    """Face kinds [axis][lo, hi], inflow state, dipole, inner sphere, floor."""
    face: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]] = ((0, 0), (0, 0), (0, 0))
    inflow: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0)  # rho, v, B(total), p
    dipole_moment: float = 0.0
    r_inner: float = 0.0
    inner: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0)   # rho, v, (B ignored), p
    p_min: float = 1e-12
    powell: int = 0

    def flat_faces(self) -> List[int]:
        return [int(self.face[d][s]) for d in range(3) for s in range(2)]


@dataclasses.dataclass
class Problem:
    name: str
    edges: List[np.ndarray]          # three ascending edge arrays
    gamma: float
    bc: BoundarySpec
    U0: np.ndarray                   # (8, nz, ny, nx) float64
    cfl: float = 0.4

    @property
    def n(self) -> Tuple[int, int, int]:
        return tuple(len(e) - 1 for e in self.edges)

    @property
    def cells(self) -> int:
        n = self.n
        return n[0] * n[1] * n[2]


# ---- grids --------------------------------------------------------------------

def uniform_axis(n: int, lo: float, hi: float) -> np.ndarray:
    return np.linspace(lo, hi, n + 1)


def _geo_count(r: float, L: float, h0: float) -> float:
    """Real-valued number of cells of widths h0 r, h0 r^2, ... covering L."""
    if L <= 0.0:
        return 0.0
    if abs(r - 1.0) < 1e-14:
        return L / h0
    return math.log1p(L * (r - 1.0) / (h0 * r)) / math.log(r)


def _geo_len(r: float, n: int, h0: float) -> float:
    if abs(r - 1.0) < 1e-14:
        return n * h0
    return h0 * r * (r ** n - 1.0) / (r - 1.0)


def _bisect(f, lo, hi, iters=200):
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def stretched_axis(n: int, lo: float, hi: float, h0: float, core: float = 10.0):
    """Edges of a stretched axis: uniform width h0 on [-core, core], geometric
    growth outward (Sec. III-B names a 1.05 ratio; with the requested cell count
    and extent one ratio per axis is solved instead so that the two stretched
    sides hold the remaining cells, then each side's ratio is re-solved so its
    last edge lands on the face).  Returns (edges, (r_lo, r_hi))."""
    c_lo, c_hi = max(lo, -core), min(hi, core)
    n_core = int(round((c_hi - c_lo) / h0))
    L_lo, L_hi = c_lo - lo, hi - c_hi
    rest = n - n_core
    if rest < 0:
        raise ValueError("core does not fit")
    if L_lo <= 0 and L_hi <= 0:
        return uniform_axis(n, lo, hi), (1.0, 1.0)
    max_cells = _geo_count(1.0, L_lo, h0) + _geo_count(1.0, L_hi, h0)
    if rest > max_cells:
        raise ValueError("too many cells for a stretched axis with this h0")
    r = _bisect(lambda r: _geo_count(r, L_lo, h0) + _geo_count(r, L_hi, h0) - rest, 1.0 + 1e-12, 4.0)
    n_lo = int(round(_geo_count(r, L_lo, h0))) if L_lo > 0 else 0
    n_hi = rest - n_lo
    if L_hi <= 0:
        n_lo, n_hi = rest, 0
    ratios = []
    sides = []
    for L, ns in ((L_lo, n_lo), (L_hi, n_hi)):
        if ns <= 0:
            ratios.append(1.0)
            sides.append(np.zeros(0))
            continue
        if ns * h0 >= L:           # uniform would already reach: shrink (rare)
            rr = 1.0
            w = np.full(ns, L / ns)
        else:
            rr = _bisect(lambda q: _geo_len(q, ns, h0) - L, 1.0 + 1e-14, 4.0)
            w = h0 * rr ** np.arange(1, ns + 1)
        ratios.append(rr)
        sides.append(w)
    core_edges = c_lo + h0 * np.arange(n_core + 1)
    core_edges[-1] = c_hi
    lo_edges = c_lo - np.cumsum(sides[0])[::-1]
    hi_edges = c_hi + np.cumsum(sides[1])
    if len(lo_edges):
        lo_edges[0] = lo
    if len(hi_edges):
        hi_edges[-1] = hi
    edges = np.concatenate([lo_edges, core_edges, hi_edges])
    assert len(edges) == n + 1
    return edges, tuple(ratios)


def centres(edges: np.ndarray) -> np.ndarray:
    return 0.5 * (edges[:-1] + edges[1:])


# ---- state helpers --------------------------------------------------------------

def conserved(rho, v, Bp, p, gamma):
    """(rho, v[3], B'[3], p) broadcast arrays -> (8, ...) conserved state."""
    rho = np.asarray(rho, dtype=np.float64)
    v = [np.asarray(c, dtype=np.float64) for c in v]
    Bp = [np.asarray(c, dtype=np.float64) for c in Bp]
    p = np.asarray(p, dtype=np.float64)
    shape = np.broadcast_shapes(rho.shape, p.shape, *[c.shape for c in v], *[c.shape for c in Bp])
    U = np.empty((8,) + shape)
    U[0] = rho
    for k in range(3):
        U[1 + k] = rho * v[k]
        U[4 + k] = Bp[k]
    U[7] = p / (gamma - 1.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) \
        + 0.5 * (Bp[0] ** 2 + Bp[1] ** 2 + Bp[2] ** 2)
    return U


def dipole_field(M, x, y, z):
    """Field of a dipole of moment M along -z at the origin (initial data only)."""
    r2 = x * x + y * y + z * z
    r = np.sqrt(r2)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r2 > 0, M / (r2 * r2 * r), 0.0)
    mr = -z
    return 3.0 * f * mr * x, 3.0 * f * mr * y, f * (3.0 * mr * z + r2)


# ---- workloads --------------------------------------------------------------------

def brio_wu_3d(n=(32, 32, 32), gamma=5.0 / 3.0) -> Problem:
    """Brio-Wu states along x on [0,1]^3, periodic, replicated in y and z."""
    nx, ny, nz = n
    edges = [uniform_axis(nx, 0.0, 1.0), uniform_axis(ny, 0.0, 1.0), uniform_axis(nz, 0.0, 1.0)]
    xc = centres(edges[0])
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    By = np.where(left, 1.0, -1.0)
    z = np.zeros(nx)
    U1 = conserved(rho, (z, z, z), (np.full(nx, 0.75), By, z), p, gamma)
    U = np.broadcast_to(U1[:, None, None, :], (8, nz, ny, nx)).copy()
    bc = BoundarySpec(face=((0, 0), (0, 0), (0, 0)))
    return Problem("brio_wu_3d", edges, gamma, bc, U, cfl=0.4)


def solar_wind(n_cc=5.0, vx_kms=-400.0, T=1.0e5, bz_nt=-5.0):
    """Solar-wind primitive state in code units [R: p = 2 n k_B T]."""
    rho = n_cc
    vx = vx_kms * 1e3 / V0
    p = 2.0 * n_cc * 1e6 * K_B * T / P_UNIT
    bz = bz_nt / B_UNIT_NT
    return rho, vx, p, bz


def dipole_moment_code() -> float:
    return B_EARTH_NT / B_UNIT_NT        # B_E R_E^3 with R_E = 1


def magnetosphere(n=(256, 192, 192), h0=0.4, n_cc=5.0, vx_kms=-400.0, T=1.0e5, bz_nt=-5.0,
                  x_ext=(-100.0, 30.0), yz_ext=(-60.0, 60.0), r_inner=3.0, gamma=5.0 / 3.0,
                  cfl=0.4, name="magnetosphere") -> Problem:
    nx, ny, nz = n
    ex, rx = stretched_axis(nx, x_ext[0], x_ext[1], h0)
    ey, ry = stretched_axis(ny, yz_ext[0], yz_ext[1], h0)
    ez, rz = stretched_axis(nz, yz_ext[0], yz_ext[1], h0)
    rho, vx, p, bz = solar_wind(n_cc, vx_kms, T, bz_nt)
    M = dipole_moment_code()
    x = centres(ex)[None, None, :]
    y = centres(ey)[None, :, None]
    z = centres(ez)[:, None, None]
    x, y, z = np.broadcast_arrays(x, y, z)
    # x <= 15: B' = field of the image dipole at (30, 0, 0); plasma at rest
    Bix, Biy, Biz = dipole_field(M, x - 30.0, y, z)
    Bdx, Bdy, Bdz = dipole_field(M, x, y, z)
    up = x > 15.0
    Bpx = np.where(up, 0.0 - Bdx, Bix)
    Bpy = np.where(up, 0.0 - Bdy, Biy)
    Bpz = np.where(up, bz - Bdz, Biz)
    vxa = np.where(up, vx, 0.0)
    zero = np.zeros_like(x)
    U = conserved(np.full_like(x, rho), (vxa, zero, zero), (Bpx, Bpy, Bpz), np.full_like(x, p), gamma)
    inside = x * x + y * y + z * z < r_inner * r_inner
    Uin = conserved(rho, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), p, gamma)
    for k in range(8):
        U[k][inside] = Uin[k]
    face = ((BC_OUTFLOW, BC_INFLOW), (BC_OUTFLOW, BC_OUTFLOW), (BC_OUTFLOW, BC_OUTFLOW))
    bc = BoundarySpec(face=face, inflow=(rho, vx, 0.0, 0.0, 0.0, 0.0, bz, p), dipole_moment=M,
                      r_inner=r_inner, inner=(rho, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, p),
                      p_min=1e-6 * p, powell=1)
    prob = Problem(name, [ex, ey, ez], gamma, bc, U, cfl=cfl)
    prob.stretch = (rx, ry, rz)
    return prob


ENSEMBLE_SEED = 160702214
ENSEMBLE_GRIDS = ((96, 96, 96), (128, 96, 96), (160, 128, 128))


def ensemble(count=48, seed=ENSEMBLE_SEED, h0=0.4) -> List[Problem]:
    """Seeded magnetosphere instances on uneven grids."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        g = ENSEMBLE_GRIDS[int(rng.integers(0, len(ENSEMBLE_GRIDS)))]
        n_cc = float(rng.uniform(2.0, 20.0))
        vx = float(rng.uniform(-800.0, -300.0))
        bz = float(rng.uniform(-10.0, 10.0))
        out.append(magnetosphere(n=g, h0=h0, n_cc=n_cc, vx_kms=vx, T=1.0e5, bz_nt=bz,
                                 name=f"ensemble[{i}]"))
    return out


# ---- 1D problems and random states for the tests ---------------------------------

def shock_tube_1d(n, left, right, gamma, x0=0.5, lo=0.0, hi=1.0, axis=0, periodic=False) -> Problem:
    """1D Riemann problem along ``axis`` (the other axes have one periodic cell).
    left/right = (rho, vn, vt1, vt2, Bn, Bt1, Bt2, p) in the local frame of the axis."""
    edges = [uniform_axis(1, 0.0, 1.0) for _ in range(3)]
    edges[axis] = uniform_axis(n, lo, hi)
    xc = centres(edges[axis])
    L, R = np.asarray(left, float), np.asarray(right, float)
    s = np.where(xc < x0, 0.0, 1.0)
    prim = L[:, None] * (1 - s) + R[:, None] * s
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    v = [None] * 3
    B = [None] * 3
    v[axis], v[t1], v[t2] = prim[1], prim[2], prim[3]
    B[axis], B[t1], B[t2] = prim[4], prim[5], prim[6]
    U1 = conserved(prim[0], v, B, prim[7], gamma)
    shape = [1, 1, 1]
    shape[axis] = n
    U = U1.reshape((8,) + tuple(reversed(shape))).copy()
    kind = BC_PERIODIC if periodic else BC_OUTFLOW
    face = [(BC_PERIODIC, BC_PERIODIC)] * 3
    face[axis] = (kind, kind)
    bc = BoundarySpec(face=tuple(face))
    return Problem("shock_tube", edges, gamma, bc, U, cfl=0.4)


def sod(n, gamma=1.4, axis=0) -> Problem:
    return shock_tube_1d(n, (1.0, 0, 0, 0, 0, 0, 0, 1.0), (0.125, 0, 0, 0, 0, 0, 0, 0.1), gamma, axis=axis)


def brio_wu_1d(n, gamma=5.0 / 3.0, axis=0) -> Problem:
    return shock_tube_1d(n, (1.0, 0, 0, 0, 0.75, 1.0, 0, 1.0), (0.125, 0, 0, 0, 0.75, -1.0, 0, 0.1), gamma,
                         axis=axis)


def alfven_wave_1d(n, eps=1e-6, gamma=5.0 / 3.0) -> Problem:
    """Linear Alfven wave on [0,1] periodic: rho = p = Bx = 1, dBy = eps sin 2 pi x,
    dvy = -dBy (right-going at v_A = 1).  Cell averages of the sine are exact."""
    e = uniform_axis(n, 0.0, 1.0)
    avg = (np.cos(2 * np.pi * e[:-1]) - np.cos(2 * np.pi * e[1:])) / (2 * np.pi * np.diff(e))
    dB = eps * avg
    one = np.ones(n)
    zero = np.zeros(n)
    U1 = conserved(one, (zero, -dB, zero), (one, dB, zero), one, gamma)
    edges = [e, uniform_axis(1, 0, 1), uniform_axis(1, 0, 1)]
    U = U1.reshape(8, 1, 1, n).copy()
    return Problem("alfven", edges, gamma, BoundarySpec(), U, cfl=0.4)


def random_smooth_state(n, seed, gamma=5.0 / 3.0, amp_v=0.3, amp_b=0.5, modes=3, edges=None):
    """Random smooth periodic state on [0,1]^3 (positive rho and p)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    if edges is None:
        edges = [uniform_axis(nx, 0, 1), uniform_axis(ny, 0, 1), uniform_axis(nz, 0, 1)]
    x = centres(edges[0])[None, None, :]
    y = centres(edges[1])[None, :, None]
    z = centres(edges[2])[:, None, None]

    def field(amp):
        f = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f = f + amp * rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * x + ky * y + kz * z) + ph)
        return f

    rho = 1.0 + 0.5 * np.abs(field(1.0)) + 0.2
    p = 1.0 + 0.5 * np.abs(field(1.0)) + 0.2
    v = [field(amp_v) for _ in range(3)]
    B = [field(amp_b) for _ in range(3)]
    return conserved(rho, v, B, p, gamma)


def random_stretched_edges(n, seed, lo=0.0, hi=1.0, jitter=0.5):
    """Ascending edges with random widths in [1-jitter, 1+jitter] x mean."""
    rng = np.random.default_rng(seed)
    w = 1.0 + jitter * rng.uniform(-1, 1, size=n)
    e = np.concatenate([[0.0], np.cumsum(w)])
    e = lo + (hi - lo) * e / e[-1]
    return e
