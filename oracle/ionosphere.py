"""Ionosphere shell of the magnetosphere model, plain numpy.

TEST INFRASTRUCTURE ONLY: part of the oracle the GPU library is checked
against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may use it; the GPU library neither imports nor calls it, and the two share
no code or table.

What it computes (Sec. II): a thin conducting shell at r_iono (110 km altitude,
1.017 R_E) closes the field-aligned currents of the magnetosphere; it is linked
to the magnetospheric inner boundary (r_inner = 3 R_E) by dipole field lines.
An electrostatic potential equation is solved on the shell and the potential,
carried along the field lines, sets the flow on the inner boundary.  The paper
gives no further equations; the readings below (marked [R]) are the ones
listed in the design notes.

  [R1] Source: the current density J = curl B' (mu0 = 1; the dipole is curl
       free) at the cell centres by centred differences over the centre-to-
       centre span, sampled at the mapping sphere r_fac by trilinear
       interpolation of the cell-centred J and B'; the parallel component is
       J . B / |B| with B = B' + B_d (B_d exact at the point).
  [R2] Mapping down a flux tube: J_par scales with |B_d| (no cross-field
       current), J_par(iono) = J_par(r_fac) |B_d(iono)| / |B_d(r_fac)|; the
       shell takes the radial component J_r = J_par(iono) B_r / |B| at the
       foot point.  Shell nodes whose field line closes below r_fac get 0.
  [R3] Potential: Sigma_P Laplacian_S Phi = J_r on the shell (uniform Pedersen
       conductance, Hall conductance neglected; sheet-current continuity
       div K = -J_r with K = -Sigma_P grad Phi), on each polar cap
       0 <= theta <= theta_max separately (theta measured from the cap's own
       pole), sin^2 theta_max = r_iono / r_inner (the foot of the field line
       through the inner boundary's equator), Phi = 0 at theta_max.
  [R4] Discretisation: cell-centred colatitudes theta_j = (j + 1/2) dtheta,
       longitudes phi_k = k dphi; the conservative five-point form of the
       spherical Laplacian (no flux through the pole), the Dirichlet edge by
       the odd ghost Phi_{n_theta} = -Phi_{n_theta - 1}.
  [R5] Back to the inner boundary: Phi is constant along dipole field lines
       (sin^2 theta / r constant); a point maps to the cap of its own hemisphere
       (z >= 0: north); outside the caps, or where the line does not reach the
       shell, Phi = 0.  On the caps Phi is interpolated bilinearly in
       (theta, phi), with the ring mean at the pole and 0 at theta_max.
  [R6] Inner-boundary flow: v = E x B_d / |B_d|^2, E = -grad Phi by centred
       differences of Phi at the neighbouring cell centres; density and
       pressure stay the fixed inner state, B' = 0.  One solve per full step,
       from the state at the start of the step.
"""
import math

import numpy as np


class IonoConfig:
    """Shell radius, current-mapping radius, Pedersen conductance (code units:
    mu0 v0 Sigma_SI) and the cap grid of each hemisphere."""

    def __init__(self, r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=24, n_phi=48):
        self.r_iono = float(r_iono)
        self.r_fac = float(r_fac)
        self.sigma_p = float(sigma_p)
        self.n_theta = int(n_theta)
        self.n_phi = int(n_phi)


def dipole(M, x, y, z):
    """Earth dipole along -z: B_d = M (3 (m.r) r - m r^2) / r^5 with m = -z
    (0 at the origin)."""
    x, y, z = (np.asarray(a, float) for a in (x, y, z))
    r2 = x * x + y * y + z * z
    safe = np.where(r2 > 0.0, r2, 1.0)
    r5 = safe * safe * np.sqrt(safe)
    mr = -z
    f = np.where(r2 > 0.0, M / r5, 0.0)
    return f * 3.0 * mr * x, f * 3.0 * mr * y, f * (3.0 * mr * z + r2)


def cap_edge(r_iono, r_inner):
    """Colatitude of the caps' low-latitude edge [R3]."""
    return math.asin(math.sqrt(r_iono / r_inner))


def cap_grid(cfg, theta_max):
    """Cell-centred colatitudes and longitudes of one cap [R4]."""
    dth = theta_max / cfg.n_theta
    dph = 2.0 * math.pi / cfg.n_phi
    th = (np.arange(cfg.n_theta) + 0.5) * dth
    ph = np.arange(cfg.n_phi) * dph
    return th, ph, dth, dph


def foot(x, y, z, r_iono):
    """Foot point of the dipole field line through (x, y, z) on the shell:
    (hemisphere 0 north / 1 south, colatitude from that pole, longitude,
    valid) [R5]."""
    x, y, z = (np.asarray(a, float) for a in (x, y, z))
    r2 = x * x + y * y + z * z
    r = np.sqrt(r2)
    s2 = np.where(r2 > 0.0, (x * x + y * y) / np.where(r2 > 0.0, r2, 1.0), 0.0)
    s2i = np.where(r > 0.0, r_iono / np.where(r > 0.0, r, 1.0), np.inf) * s2
    valid = (r > 0.0) & (s2i <= 1.0)
    th = np.arcsin(np.sqrt(np.clip(s2i, 0.0, 1.0)))
    ph = np.mod(np.arctan2(y, x), 2.0 * math.pi)
    hemi = np.where(z >= 0.0, 0, 1)
    return hemi, th, ph, valid


def cell_centres(edges):
    return [0.5 * (np.asarray(e)[1:] + np.asarray(e)[:-1]) for e in edges]


def curl(U, centres):
    """J = curl B' at the cell centres (NaN on the outermost cells of each
    axis, which have no centred difference) [R1].  U: (8, nz, ny, nx)."""
    cx, cy, cz = centres
    B = [U[4], U[5], U[6]]

    def ddx(f, c, ax):
        out = np.full(f.shape, np.nan)
        sl_p = [slice(None)] * 3
        sl_m = [slice(None)] * 3
        sl_c = [slice(None)] * 3
        sl_p[ax], sl_m[ax], sl_c[ax] = slice(2, None), slice(None, -2), slice(1, -1)
        span = c[2:] - c[:-2]
        shape = [1, 1, 1]
        shape[ax] = span.size
        out[tuple(sl_c)] = (f[tuple(sl_p)] - f[tuple(sl_m)]) / span.reshape(shape)
        return out

    # array axes: 0 = z, 1 = y, 2 = x
    dBz_dy, dBy_dz = ddx(B[2], cy, 1), ddx(B[1], cz, 0)
    dBx_dz, dBz_dx = ddx(B[0], cz, 0), ddx(B[2], cx, 2)
    dBy_dx, dBx_dy = ddx(B[1], cx, 2), ddx(B[0], cy, 1)
    return dBz_dy - dBy_dz, dBx_dz - dBz_dx, dBy_dx - dBx_dy


def trilinear(fields, centres, x, y, z):
    """Trilinear interpolation of cell-centred fields at the points (x, y, z)."""
    cx, cy, cz = centres
    out = []
    idx = []
    for c, p in ((cx, x), (cy, y), (cz, z)):
        i = np.clip(np.searchsorted(c, p, side="right") - 1, 0, c.size - 2)
        t = (p - c[i]) / (c[i + 1] - c[i])
        idx.append((i, t))
    (ix, tx), (iy, ty), (iz, tz) = idx
    for f in fields:
        v = 0.0
        for dz in (0, 1):
            wz = tz if dz else 1.0 - tz
            for dy in (0, 1):
                wy = ty if dy else 1.0 - ty
                for dx in (0, 1):
                    wx = tx if dx else 1.0 - tx
                    v = v + wz * wy * wx * f[iz + dz, iy + dy, ix + dx]
        out.append(v)
    return out


def radial_current(U, edges, M, r_inner, cfg):
    """J_r on the two caps, shape (2, n_theta, n_phi) [R1, R2]."""
    centres = cell_centres(edges)
    J = curl(U, centres)
    theta_max = cap_edge(cfg.r_iono, r_inner)
    th, ph, _, _ = cap_grid(cfg, theta_max)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    out = np.zeros((2, cfg.n_theta, cfg.n_phi))
    for h in (0, 1):
        zs = 1.0 if h == 0 else -1.0
        s2m = (cfg.r_fac / cfg.r_iono) * np.sin(TH) ** 2          # sin^2 at r_fac on the same line
        reach = s2m <= 1.0
        thm = np.arcsin(np.sqrt(np.clip(s2m, 0.0, 1.0)))
        px = cfg.r_fac * np.sin(thm) * np.cos(PH)
        py = cfg.r_fac * np.sin(thm) * np.sin(PH)
        pz = zs * cfg.r_fac * np.cos(thm)
        Jx, Jy, Jz, Bx, By, Bz = trilinear(list(J) + [U[4], U[5], U[6]], centres, px, py, pz)
        dx, dy, dz = dipole(M, px, py, pz)
        Bx, By, Bz = Bx + dx, By + dy, Bz + dz
        jpar = (Jx * Bx + Jy * By + Jz * Bz) / np.sqrt(Bx * Bx + By * By + Bz * Bz)
        # foot point on the shell
        fx = cfg.r_iono * np.sin(TH) * np.cos(PH)
        fy = cfg.r_iono * np.sin(TH) * np.sin(PH)
        fz = zs * cfg.r_iono * np.cos(TH)
        ix_, iy_, iz_ = dipole(M, fx, fy, fz)
        bi = np.sqrt(ix_ * ix_ + iy_ * iy_ + iz_ * iz_)
        bm = np.sqrt(dx * dx + dy * dy + dz * dz)
        br = (ix_ * fx + iy_ * fy + iz_ * fz) / cfg.r_iono
        jr = jpar * (bi / bm) * (br / bi)
        out[h] = np.where(reach, jr, 0.0)
    return out


def laplacian_matrix(cfg, theta_max):
    """The discrete cap operator of [R4] on the unit sphere, rows and columns
    ordered (j, k) with k fastest."""
    th, _, dth, dph = cap_grid(cfg, theta_max)
    nt, npp = cfg.n_theta, cfg.n_phi
    A = np.zeros((nt * npp, nt * npp))
    for j in range(nt):
        s = math.sin(th[j])
        sp = math.sin(th[j] + 0.5 * dth)
        sm = math.sin(th[j] - 0.5 * dth) if j > 0 else 0.0
        for k in range(npp):
            row = j * npp + k
            A[row, row] -= (sp + sm) / (s * dth * dth)
            if j + 1 < nt:
                A[row, (j + 1) * npp + k] += sp / (s * dth * dth)
            else:
                A[row, row] -= sp / (s * dth * dth)       # odd ghost: Phi = 0 at theta_max
            if j > 0:
                A[row, (j - 1) * npp + k] += sm / (s * dth * dth)
            A[row, j * npp + (k + 1) % npp] += 1.0 / (s * s * dph * dph)
            A[row, j * npp + (k - 1) % npp] += 1.0 / (s * s * dph * dph)
            A[row, row] -= 2.0 / (s * s * dph * dph)
    return A


def solve_potential(jr, r_inner, cfg):
    """Phi on the two caps from Sigma_P Laplacian Phi = J_r [R3, R4]."""
    theta_max = cap_edge(cfg.r_iono, r_inner)
    A = laplacian_matrix(cfg, theta_max)
    phi = np.zeros_like(jr)
    for h in (0, 1):
        rhs = (cfg.r_iono * cfg.r_iono / cfg.sigma_p) * jr[h].reshape(-1)
        phi[h] = np.linalg.solve(A, rhs).reshape(cfg.n_theta, cfg.n_phi)
    return phi


def potential_at(phi, x, y, z, r_inner, cfg):
    """Phi carried along the dipole field lines to the points (x, y, z) [R5]."""
    theta_max = cap_edge(cfg.r_iono, r_inner)
    _, _, dth, dph = cap_grid(cfg, theta_max)
    hemi, th, ph, valid = foot(x, y, z, cfg.r_iono)
    inside = valid & (th < theta_max)
    nt, npp = cfg.n_theta, cfg.n_phi
    t = th / dth - 0.5                      # ring position (ring j at t = j)
    u = ph / dph
    k0 = np.floor(u).astype(int) % npp
    k1 = (k0 + 1) % npp
    fu = u - np.floor(u)
    out = np.zeros(np.shape(th))
    for idx in np.ndindex(np.shape(th)):
        if not inside[idx]:
            continue
        P = phi[hemi[idx]]

        def ring(j):
            if j < 0:
                return P[0].mean()          # the pole
            if j >= nt:
                return 0.0                  # the cap edge
            return (1.0 - fu[idx]) * P[j, k0[idx]] + fu[idx] * P[j, k1[idx]]

        tt = t[idx]
        if tt < 0.0:                        # between the pole (t = -1/2) and ring 0
            w = (tt + 0.5) / 0.5
            out[idx] = (1.0 - w) * ring(-1) + w * ring(0)
        elif tt > nt - 1:                   # between the last ring and the edge (t = n - 1/2)
            w = (tt - (nt - 1)) / 0.5
            out[idx] = (1.0 - w) * ring(nt - 1) + w * 0.0
        else:
            j = int(math.floor(tt))
            w = tt - j
            out[idx] = (1.0 - w) * ring(j) + w * ring(j + 1)
    return out


def inner_drift(phi, edges, M, r_inner, cfg):
    """E = -grad Phi and v = E x B_d / |B_d|^2 on the cells inside the inner
    sphere, each (3, nz, ny, nx), zero elsewhere [R6]."""
    cx, cy, cz = cell_centres(edges)
    nx, ny, nz = cx.size, cy.size, cz.size
    E = np.zeros((3, nz, ny, nx))
    v = np.zeros((3, nz, ny, nx))
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    iz, iy, ix = np.nonzero(X * X + Y * Y + Z * Z < r_inner * r_inner)
    if iz.size == 0:
        return E, v
    x, y, z = cx[ix], cy[iy], cz[iz]
    for d, (c, i, n) in enumerate(((cx, ix, nx), (cy, iy, ny), (cz, iz, nz))):
        lo, hi = np.maximum(i - 1, 0), np.minimum(i + 1, n - 1)
        pm = [x.copy(), y.copy(), z.copy()]
        pp = [x.copy(), y.copy(), z.copy()]
        pm[d], pp[d] = c[lo], c[hi]
        fm = potential_at(phi, pm[0], pm[1], pm[2], r_inner, cfg)
        fp = potential_at(phi, pp[0], pp[1], pp[2], r_inner, cfg)
        E[d, iz, iy, ix] = -(fp - fm) / (c[hi] - c[lo])
    bx, by, bz = dipole(M, x, y, z)
    b2 = bx * bx + by * by + bz * bz
    ok = b2 > 0.0
    b2 = np.where(ok, b2, 1.0)
    Ex, Ey, Ez = E[0, iz, iy, ix], E[1, iz, iy, ix], E[2, iz, iy, ix]
    v[0, iz, iy, ix] = np.where(ok, (Ey * bz - Ez * by) / b2, 0.0)
    v[1, iz, iy, ix] = np.where(ok, (Ez * bx - Ex * bz) / b2, 0.0)
    v[2, iz, iy, ix] = np.where(ok, (Ex * by - Ey * bx) / b2, 0.0)
    return E, v


def couple(U, edges, M, r_inner, cfg):
    """One ionosphere solve: (inner-cell velocities, Phi, J_r)."""
    jr = radial_current(U, edges, M, r_inner, cfg)
    phi = solve_potential(jr, r_inner, cfg)
    return inner_drift(phi, edges, M, r_inner, cfg)[1], phi, jr
