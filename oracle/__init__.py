"""Oracle: a plain, slow FP64 CPU implementation of the split PPMLR-MHD sweep.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library and never imports it.  The arithmetic lives in
``ppmlr_oracle.c`` (see its header for what each routine restates); this module
only marshals arrays through ctypes.
"""
import ctypes
import os

import numpy as np

from .build import build, LIB

BC_PERIODIC, BC_OUTFLOW, BC_INFLOW = 0, 1, 2
FLAG_CFL, FLAG_NONFINITE = 1, 2

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("PPMLR_ORACLE_LIB")   # a planted-mistake copy (mutation tests)
        if not path:
            path = build()
        L = ctypes.CDLL(path)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int] * 3 + [_dp] * 3 + [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                 _dp, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double, ctypes.c_int]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_state.argtypes = [ctypes.c_void_p, _dp]
        L.orc_get_state.argtypes = [ctypes.c_void_p, _dp]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_sweep.restype = ctypes.c_int
        L.orc_sweep.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_floor_hits.restype = ctypes.c_longlong
        L.orc_floor_hits.argtypes = [ctypes.c_void_p]
        L.orc_step_count.restype = ctypes.c_longlong
        L.orc_step_count.argtypes = [ctypes.c_void_p]
        L.orc_set_step_count.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
        L.orc_sweep_sampled.restype = ctypes.c_int
        L.orc_sweep_sampled.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_dipole.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.orc_fast_speed2.restype = ctypes.c_double
        L.orc_fast_speed2.argtypes = [ctypes.c_double] * 6
        L.orc_ppm_edges.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp]
        L.orc_ppm_parabola.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.orc_avg_right.restype = ctypes.c_double
        L.orc_avg_right.argtypes = [ctypes.c_double] * 4
        L.orc_avg_left.restype = ctypes.c_double
        L.orc_avg_left.argtypes = [ctypes.c_double] * 4
        L.orc_riemann.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_riemann_nl.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp]
        L.orc_set_riemann.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_steepening.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_inner_velocity.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_flatten.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count in use."""
    return lib().orc_set_threads(int(n))


class Oracle:
    """One grid and boundary specification, state held on the host.

    edges: three ascending arrays of n[d]+1 cell edges.  bc: six face kinds
    (x lo, x hi, y lo, y hi, z lo, z hi).  inflow / inner: (rho, vx, vy, vz,
    Bx, By, Bz, p); inflow B is the total field, inner B is ignored (B' = 0).
    State arrays are (8, nz, ny, nx): rho, m_x, m_y, m_z, B'_x, B'_y, B'_z, E.
    """

    def __init__(self, edges, gamma, bc, inflow=None, dipole_moment=0.0, r_inner=0.0,
                 inner=None, p_min=1e-12, powell=0):
        L = lib()
        self.edges = [np.ascontiguousarray(e, dtype=np.float64) for e in edges]
        self.n = tuple(len(e) - 1 for e in self.edges)
        bc_arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
        infl = np.ascontiguousarray(inflow if inflow is not None else np.zeros(8), dtype=np.float64)
        inn = np.ascontiguousarray(inner if inner is not None else np.zeros(8), dtype=np.float64)
        self._h = L.orc_create(self.n[0], self.n[1], self.n[2], _ptr(self.edges[0]), _ptr(self.edges[1]),
                               _ptr(self.edges[2]), float(gamma), bc_arr, _ptr(infl), float(dipole_moment),
                               float(r_inner), _ptr(inn), float(p_min), int(powell))
        if not self._h:
            raise ValueError("oracle: invalid grid")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (8, self.n[2], self.n[1], self.n[0])

    def set_state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == self.shape
        lib().orc_set_state(self._h, _ptr(U))

    def get_state(self):
        U = np.empty(self.shape, dtype=np.float64)
        lib().orc_get_state(self._h, _ptr(U))
        return U

    def cfl_dt(self, cfl):
        return lib().orc_cfl_dt(self._h, float(cfl))

    def step(self, dt):
        return lib().orc_step(self._h, float(dt))

    def sweep(self, axis, dt):
        return lib().orc_sweep(self._h, int(axis), float(dt))

    def sweep_sampled(self, axis, dt, j, k):
        """One sweep of the listed pencils only (state unchanged); returns
        (npencil, 8, n[axis]) and the flags."""
        j = np.ascontiguousarray(j, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        out = np.empty((len(j), 8, self.n[axis]))
        ip = ctypes.POINTER(ctypes.c_int)
        fl = lib().orc_sweep_sampled(self._h, int(axis), float(dt), len(j), j.ctypes.data_as(ip),
                                     k.ctypes.data_as(ip), _ptr(out))
        return out, fl

    @property
    def floor_hits(self):
        return lib().orc_floor_hits(self._h)

    @property
    def step_count(self):
        return lib().orc_step_count(self._h)

    @step_count.setter
    def step_count(self, s):
        lib().orc_set_step_count(self._h, int(s))

    def set_inner_velocity(self, v):
        """Flow of the inner-sphere cells, (3, nz, ny, nx) or None (the fixed
        inner state's own flow)."""
        if v is None:
            lib().orc_set_inner_velocity(self._h, None)
            return
        a = np.ascontiguousarray(v, dtype=np.float64)
        lib().orc_set_inner_velocity(self._h, a.ctypes.data_as(ctypes.c_void_p))

    def set_steepening(self, on):
        """Contact steepening of the remapped densities (Colella & Woodward 1984)."""
        lib().orc_set_steepening(self._h, int(bool(on)))

    def set_riemann(self, iters):
        """0: two-wave Riemann solver; k > 0: k two-shock Newton steps on the
        fast mode (nonlinear variant)."""
        lib().orc_set_riemann(self._h, int(iters))

    def run(self, cfl, nsteps=None, t_end=None, max_steps=10**7):
        """Advance with the CFL time step for nsteps steps or up to t_end."""
        t, k, flags = 0.0, 0, 0
        while True:
            if nsteps is not None and k >= nsteps:
                break
            if t_end is not None and t >= t_end * (1 - 1e-14):
                break
            if k >= max_steps:
                raise RuntimeError("oracle: too many steps")
            dt = self.cfl_dt(cfl)
            if t_end is not None and t + dt > t_end:
                dt = t_end - t
            flags |= self.step(dt)
            t += dt
            k += 1
        return t, k, flags


# ---- unit-level routines (for the pins) -------------------------------------

def dipole(M, x, y, z):
    out = np.zeros(3)
    lib().orc_dipole(float(M), float(x), float(y), float(z), _ptr(out))
    return out


def fast_speed2(rho, p, Bn, B1, B2, gamma):
    return lib().orc_fast_speed2(float(rho), float(p), float(Bn), float(B1), float(B2), float(gamma))


def ppm_edges(xi, a, limited=True):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_ppm_edges(len(a), _ptr(xi), _ptr(a), int(bool(limited)), _ptr(out))
    return out


def ppm_parabola(ai, aL, aR, f=0.0):
    out = np.zeros(3)
    lib().orc_ppm_parabola(float(ai), float(aL), float(aR), float(f), _ptr(out))
    return out


def flatten(Pt, u):
    """Flattening of a pencil from its total pressure and normal velocity
    (Colella & Woodward 1984, App. A): returns (ft, f); ft is the shock
    indicator of every zone (0 outside 2..n-3), f the coefficient of zones
    3..n-4 (0 elsewhere)."""
    Pt = np.ascontiguousarray(Pt, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert Pt.shape == u.shape and Pt.ndim == 1
    ft = np.zeros_like(Pt)
    f = np.zeros_like(Pt)
    lib().orc_flatten(len(Pt), _ptr(Pt), _ptr(u), _ptr(ft), _ptr(f))
    return ft, f


def avg_right(aL, aR, a6, y):
    return lib().orc_avg_right(float(aL), float(aR), float(a6), float(y))


def avg_left(aL, aR, a6, y):
    return lib().orc_avg_left(float(aL), float(aR), float(a6), float(y))


def riemann(L, R, Bn, gamma, iters=0):
    """L, R = (rho, u, v1, v2, B1, B2, p[, B1a, B2a]); when the Alfven-traced
    B1a, B2a are omitted they equal B1, B2.  iters = 0: two-wave solver;
    iters > 0: that many two-shock Newton steps on the fast mode.  Returns
    (u*, P*, S*, v1*, v2*, sigma1*, sigma2*, F_E)."""
    def full(s):
        s = list(map(float, s))
        if len(s) == 7:
            s = s + s[4:6]
        return np.ascontiguousarray(s, dtype=np.float64)
    Lv, Rv = full(L), full(R)
    out = np.zeros(8)
    lib().orc_riemann_nl(_ptr(Lv), _ptr(Rv), float(Bn), float(gamma), int(iters), _ptr(out))
    return out
