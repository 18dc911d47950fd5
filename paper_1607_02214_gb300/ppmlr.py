"""ctypes binding of the C ABI in include/ppmlr.h (argument marshalling only).

Every function of the ABI is exposed under its own name; ``Context`` bundles
them for torch tensors and numpy arrays.  All arithmetic runs in the CUDA
library libppmlr_gb300.so; there is no CPU fallback: loading fails loudly if
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PPMLR_LIBRARY selects another build of the same library (the bounds-checked
# build the tests make with build.build(check=True)).
LIB_PATH = os.environ.get("PPMLR_LIBRARY", os.path.join(HERE, "libppmlr_gb300.so"))

(PPMLR_OK, PPMLR_E_INVALID, PPMLR_E_CUDA, PPMLR_E_OOM, PPMLR_E_NONFINITE, PPMLR_E_CFL, PPMLR_E_TIMEOUT,
 PPMLR_E_BOUNDS) = range(8)
PPMLR_FP64, PPMLR_MIXED, PPMLR_FP64_EXACT = 0, 1, 2
PPMLR_BC_PERIODIC, PPMLR_BC_OUTFLOW, PPMLR_BC_INFLOW = 0, 1, 2
STATUS_NAMES = {0: "PPMLR_OK", 1: "PPMLR_E_INVALID", 2: "PPMLR_E_CUDA", 3: "PPMLR_E_OOM",
                4: "PPMLR_E_NONFINITE", 5: "PPMLR_E_CFL", 6: "PPMLR_E_TIMEOUT", 7: "PPMLR_E_BOUNDS"}


class ppmlr_grid(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("edges", POINTER(c_double) * 3)]


class ppmlr_prim(ctypes.Structure):
    _fields_ = [("rho", c_double), ("v", c_double * 3), ("B", c_double * 3), ("p", c_double)]


class ppmlr_bc(ctypes.Structure):
    _fields_ = [("face", (c_int * 2) * 3), ("inflow", ppmlr_prim), ("dipole_moment", c_double),
                ("r_inner", c_double), ("inner", ppmlr_prim), ("p_min", c_double), ("powell", c_int)]


class ppmlr_iono(ctypes.Structure):
    _fields_ = [("r_iono", c_double), ("r_fac", c_double), ("sigma_p", c_double), ("n_theta", c_int),
                ("n_phi", c_int)]


DPTR8 = POINTER(c_double) * 8

# (name, restype, argtypes) of every exported function
SIGNATURES = [
    ("ppmlr_create", c_int, [POINTER(ppmlr_grid), c_double, POINTER(ppmlr_bc), c_int, c_void_p, POINTER(c_void_p)]),
    ("ppmlr_set_stream", c_int, [c_void_p, c_void_p]),
    ("ppmlr_set_state", c_int, [c_void_p, DPTR8, c_int]),
    ("ppmlr_get_state", c_int, [c_void_p, DPTR8, c_int]),
    ("ppmlr_get_layers", c_int, [c_void_p, c_int, c_int, DPTR8, c_int]),
    ("ppmlr_set_layers", c_int, [c_void_p, c_int, c_int, DPTR8, c_int]),
    ("ppmlr_cfl_dt", c_int, [c_void_p, c_double, POINTER(c_double)]),
    ("ppmlr_step", c_int, [c_void_p, c_double]),
    ("ppmlr_step_cfl", c_int, [c_void_p, c_double, c_int]),
    ("ppmlr_sweep", c_int, [c_void_p, c_int, c_double]),
    ("ppmlr_check", c_int, [c_void_p]),
    ("ppmlr_get_diagnostics", c_int, [c_void_p, POINTER(c_longlong), POINTER(c_longlong), POINTER(c_int)]),
    ("ppmlr_set_step_count", c_int, [c_void_p, c_longlong]),
    ("ppmlr_get_dt", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_last_error", ctypes.c_char_p, [c_void_p]),
    ("ppmlr_destroy", None, [c_void_p]),
    ("ppmlr_launch_count", c_longlong, [c_void_p]),
    ("ppmlr_enable_timing", c_int, [c_void_p, c_int]),
    ("ppmlr_read_timing", c_int, [c_void_p, POINTER(c_double), POINTER(c_longlong)]),
    ("ppmlr_autotune", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_get_tiles", c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    ("ppmlr_get_sweep_forms", c_int, [c_void_p, POINTER(c_int)]),
    ("ppmlr_set_sweep_form", c_int, [c_void_p, c_int, c_int]),
    ("ppmlr_set_tiles", c_int, [c_void_p, c_int, c_int, c_int]),
    ("ppmlr_run", c_int, [c_void_p, c_double, c_longlong, c_int]),
    ("ppmlr_set_riemann_solver", c_int, [c_void_p, c_int]),
    ("ppmlr_set_steepening", c_int, [c_void_p, c_int]),
    ("ppmlr_selftest_wait_timeout", c_int, [c_void_p]),
    ("ppmlr_set_ionosphere", c_int, [c_void_p, POINTER(ppmlr_iono)]),
    ("ppmlr_ionosphere_solve", c_int, [c_void_p]),
    ("ppmlr_get_ionosphere", c_int, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    ("ppmlr_ensemble_set_steepening", c_int, [c_void_p, c_int]),
    ("ppmlr_get_time", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_set_time", c_int, [c_void_p, c_double]),
    ("ppmlr_checkpoint_save", c_int, [c_void_p, ctypes.c_char_p]),
    ("ppmlr_checkpoint_load", c_int, [c_void_p, ctypes.c_char_p]),
    ("ppmlr_checkpoint_info", c_int, [ctypes.c_char_p, POINTER(c_int), POINTER(c_longlong), POINTER(c_double),
                                      POINTER(c_int)]),
    ("ppmlr_ensemble_create", c_int, [c_int, POINTER(ppmlr_grid), POINTER(ppmlr_bc), c_double, c_int, c_void_p,
                                      POINTER(c_void_p)]),
    ("ppmlr_ensemble_set_stream", c_int, [c_void_p, c_void_p]),
    ("ppmlr_ensemble_set_state", c_int, [c_void_p, c_int, DPTR8, c_int]),
    ("ppmlr_ensemble_get_state", c_int, [c_void_p, c_int, DPTR8, c_int]),
    ("ppmlr_ensemble_step", c_int, [c_void_p, c_double, c_int]),
    ("ppmlr_ensemble_time_kernels", c_int, [c_void_p, c_double, c_int, POINTER(c_double)]),
    ("ppmlr_ensemble_autotune", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_ensemble_get_tiles", c_int, [c_void_p, POINTER(c_int)]),
    ("ppmlr_ensemble_set_riemann_solver", c_int, [c_void_p, c_int]),
    ("ppmlr_ensemble_set_launch", c_int, [c_void_p, c_int, c_int, c_int]),
    ("ppmlr_ensemble_get_dt", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_ensemble_check", c_int, [c_void_p]),
    ("ppmlr_ensemble_get_diagnostics", c_int, [c_void_p, POINTER(c_longlong), POINTER(c_longlong)]),
    ("ppmlr_ensemble_last_error", ctypes.c_char_p, [c_void_p]),
    ("ppmlr_ensemble_launch_count", c_longlong, [c_void_p]),
    ("ppmlr_ensemble_destroy", None, [c_void_p]),
    ("ppmlr_cfl_dt_noalloc", c_int, [DPTR8, POINTER(c_int), POINTER(c_double) * 3, POINTER(c_double) * 3,
                                     c_double, c_double, c_double, c_double, c_double, c_int, POINTER(c_double),
                                     c_void_p]),
    ("ppmlr_measure_pipe_rates", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_selftest_fp64_arith", c_int, [c_void_p, c_longlong, POINTER(c_double)]),
    ("ppmlr_measure_coissue", c_int, [c_void_p, POINTER(c_double)]),
    ("ppmlr_set_march_chunk", c_int, [c_void_p, c_int, c_int]),
]

_lib = None


def load():
    """Load libppmlr_gb300.so (raises if it is missing: no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def __getattr__(name):          # module-level access to the raw ABI functions
    if name.startswith("ppmlr_"):
        return getattr(load(), name)
    raise AttributeError(name)


def measure_pipe_rates(stream=None):
    """Instructions per second of FP64 FMA, FP64 add and FP32 FMA on the
    current GPU (ppmlr_measure_pipe_rates)."""
    out = (c_double * 3)()
    st = load().ppmlr_measure_pipe_rates(c_void_p(stream), out)
    if st != PPMLR_OK:
        raise PPMLRError(st, "ppmlr_measure_pipe_rates failed")
    return {"dfma_per_s": out[0], "dadd_per_s": out[1], "ffma_per_s": out[2]}


def measure_coissue(stream=None):
    """Integer-pipe double products per second alone, and FP64 FMAs plus
    such products per second when interleaved (ppmlr_measure_coissue)."""
    out = (c_double * 2)()
    st = load().ppmlr_measure_coissue(c_void_p(stream), out)
    if st != PPMLR_OK:
        raise PPMLRError(st, "ppmlr_measure_coissue failed")
    return {"int_dmul_per_s": out[0], "dfma_plus_int_dmul_per_s": out[1]}


def selftest_fp64_arith(n=1 << 22, stream=None):
    """Largest error, in ulps of the correctly rounded result, of the
    PPMLR_FP64 form's square root and reciprocal over n arguments spanning
    2^-1000..2^1000, how many of the square roots differ from the correctly
    rounded ones, and how many of n products on the integer pipes differ
    from the IEEE products (ppmlr_selftest_fp64_arith)."""
    out = (c_double * 4)()
    st = load().ppmlr_selftest_fp64_arith(c_void_p(stream), n, out)
    if st != PPMLR_OK:
        raise PPMLRError(st, "ppmlr_selftest_fp64_arith failed")
    return {"sqrt_ulp": out[0], "recip_ulp": out[1], "sqrt_mismatches": int(out[2]),
            "mul_mismatches": int(out[3])}


class PPMLRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _prim(vals):
    p = ppmlr_prim()
    p.rho = vals[0]
    for k in range(3):
        p.v[k] = vals[1 + k]
        p.B[k] = vals[4 + k]
    p.p = vals[7]
    return p


def make_bc(spec) -> ppmlr_bc:
    """ppmlr_bc from an inputs.BoundarySpec-like object."""
    bc = ppmlr_bc()
    for d in range(3):
        for s in range(2):
            bc.face[d][s] = int(spec.face[d][s])
    bc.inflow = _prim(spec.inflow)
    bc.dipole_moment = float(spec.dipole_moment)
    bc.r_inner = float(spec.r_inner)
    bc.inner = _prim(spec.inner)
    bc.p_min = float(spec.p_min)
    bc.powell = int(spec.powell)
    return bc


def _stream_handle(stream):
    if stream is None:
        import torch
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


class Context:
    """One grid + boundary spec + state on the current CUDA device."""

    def __init__(self, edges, gamma, bc_spec, precision=PPMLR_FP64, stream=None):
        L = load()
        self._edges = [np.ascontiguousarray(e, dtype=np.float64) for e in edges]
        self.n = tuple(len(e) - 1 for e in self._edges)
        g = ppmlr_grid()
        for d in range(3):
            g.n[d] = self.n[d]
            g.edges[d] = self._edges[d].ctypes.data_as(POINTER(c_double))
        self._bc = make_bc(bc_spec)
        h = c_void_p()
        st = L.ppmlr_create(ctypes.byref(g), float(gamma), ctypes.byref(self._bc), int(precision),
                            _stream_handle(stream), ctypes.byref(h))
        if st != PPMLR_OK:
            raise PPMLRError(st, "ppmlr_create failed")
        self._h = h
        self.precision = precision

    @classmethod
    def from_problem(cls, prob, precision=PPMLR_FP64, stream=None):
        return cls(prob.edges, prob.gamma, prob.bc, precision, stream)

    def close(self):
        if getattr(self, "_h", None):
            load().ppmlr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (8, self.n[2], self.n[1], self.n[0])

    def _check(self, st):
        if st != PPMLR_OK:
            raise PPMLRError(st, load().ppmlr_last_error(self._h).decode())
        return st

    def status(self, st):
        """Return the status code without raising."""
        return st

    @staticmethod
    def _ptrs(arr):
        arr8 = DPTR8()
        if hasattr(arr, "data_ptr"):
            assert arr.is_contiguous() and arr.dtype.__str__() == "torch.float64"
            step = arr[0].numel() * 8
            base = arr.data_ptr()
            for v in range(8):
                arr8[v] = ctypes.cast(c_void_p(base + v * step), POINTER(c_double))
            return arr8, 1
        assert arr.flags["C_CONTIGUOUS"] and arr.dtype == np.float64
        for v in range(8):
            arr8[v] = arr[v].ctypes.data_as(POINTER(c_double))
        return arr8, 0

    def set_state(self, U, raise_on_error=True):
        if not hasattr(U, "data_ptr"):
            U = np.ascontiguousarray(U, dtype=np.float64)
        assert tuple(U.shape) == self.shape
        p, dev = self._ptrs(U)
        st = load().ppmlr_set_state(self._h, p, dev)
        return self._check(st) if raise_on_error else st

    def get_state(self, out=None, raise_on_error=True):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        p, dev = self._ptrs(out)
        st = load().ppmlr_get_state(self._h, p, dev)
        if raise_on_error:
            self._check(st)
            return out
        return out, st

    def get_layers(self, k0, nk, out=None):
        """z layers k0 .. k0+nk-1 of the state, (8, nk, ny, nx): into `out`
        (a contiguous float64 numpy array or device tensor) or a new numpy
        array."""
        if out is None:
            out = np.empty((8, nk, self.shape[2], self.shape[3]), dtype=np.float64)
        assert tuple(out.shape) == (8, nk, self.shape[2], self.shape[3])
        p, dev = self._ptrs(out)
        self._check(load().ppmlr_get_layers(self._h, int(k0), int(nk), p, dev))
        return out

    def set_layers(self, k0, U):
        """Overwrite z layers k0 .. k0+len-1 with U, (8, nk, ny, nx)."""
        if not hasattr(U, "data_ptr"):
            U = np.ascontiguousarray(U, dtype=np.float64)
        assert tuple(U.shape)[0] == 8 and tuple(U.shape)[2:] == self.shape[2:]
        p, dev = self._ptrs(U)
        return self._check(load().ppmlr_set_layers(self._h, int(k0), int(U.shape[1]), p, dev))

    def cfl_dt(self, cfl):
        dt = c_double()
        self._check(load().ppmlr_cfl_dt(self._h, float(cfl), ctypes.byref(dt)))
        return dt.value

    def step(self, dt, raise_on_error=True):
        st = load().ppmlr_step(self._h, float(dt))
        return self._check(st) if raise_on_error else st

    def step_cfl(self, cfl, nsteps=1):
        return self._check(load().ppmlr_step_cfl(self._h, float(cfl), int(nsteps)))

    def sweep(self, axis, dt):
        return self._check(load().ppmlr_sweep(self._h, int(axis), float(dt)))

    def check(self, raise_on_error=True):
        st = load().ppmlr_check(self._h)
        return self._check(st) if raise_on_error else st

    def diagnostics(self):
        s, f, o = c_longlong(), c_longlong(), c_int()
        self._check(load().ppmlr_get_diagnostics(self._h, ctypes.byref(s), ctypes.byref(f), ctypes.byref(o)))
        return {"step": s.value, "floor_hits": f.value, "order_parity": o.value}

    def set_step_count(self, step):
        return self._check(load().ppmlr_set_step_count(self._h, int(step)))

    def last_dt(self):
        dt = c_double()
        self._check(load().ppmlr_get_dt(self._h, ctypes.byref(dt)))
        return dt.value

    def set_riemann_solver(self, iters):
        """0: two-wave Riemann solver; k > 0: k two-shock Newton steps on the
        fast mode (nonlinear variant)."""
        return self._check(load().ppmlr_set_riemann_solver(self._h, int(iters)))

    def set_steepening(self, on):
        """Contact steepening of the remapped densities (default off)."""
        return self._check(load().ppmlr_set_steepening(self._h, int(bool(on))))

    def set_ionosphere(self, r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=24, n_phi=48, on=True):
        """Ionosphere shell coupled to the inner boundary (on=False: off).
        sigma_p in code units (mu0 v0 Sigma_SI: 0.6283 is 5 S)."""
        if not on:
            return self._check(load().ppmlr_set_ionosphere(self._h, None))
        cfg = ppmlr_iono(float(r_iono), float(r_fac), float(sigma_p), int(n_theta), int(n_phi))
        self._iono = (int(n_theta), int(n_phi))
        return self._check(load().ppmlr_set_ionosphere(self._h, ctypes.byref(cfg)))

    def selftest_wait_timeout(self):
        """Launch the bounded-wait self-test (the next check reports PPMLR_E_TIMEOUT)."""
        return self._check(load().ppmlr_selftest_wait_timeout(self._h))

    def ionosphere_solve(self):
        """One shell solve from the current state (each step does one first)."""
        return self._check(load().ppmlr_ionosphere_solve(self._h))

    def get_ionosphere(self):
        """(phi, jr) of the last solve, each (2, n_theta, n_phi): north cap
        then south, colatitude rings, longitude fastest."""
        nt, npp = self._iono
        phi = np.empty((2, nt, npp))
        jr = np.empty((2, nt, npp))
        self._check(load().ppmlr_get_ionosphere(self._h, phi.ctypes.data_as(POINTER(c_double)),
                                                jr.ctypes.data_as(POINTER(c_double))))
        return phi, jr

    def run(self, cfl, nsteps, graph_steps=16):
        """nsteps device-dt steps (as step_cfl), replayed from CUDA graphs of
        graph_steps steps (0: direct launches)."""
        return self._check(load().ppmlr_run(self._h, float(cfl), int(nsteps), int(graph_steps)))

    @property
    def time(self):
        """Simulated time in code units (R_E / 100 km/s)."""
        t = c_double()
        self._check(load().ppmlr_get_time(self._h, ctypes.byref(t)))
        return t.value

    @time.setter
    def time(self, t):
        self._check(load().ppmlr_set_time(self._h, float(t)))

    def checkpoint_save(self, path):
        return self._check(load().ppmlr_checkpoint_save(self._h, os.fsencode(path)))

    def checkpoint_load(self, path):
        return self._check(load().ppmlr_checkpoint_load(self._h, os.fsencode(path)))

    @property
    def launch_count(self):
        return load().ppmlr_launch_count(self._h)

    def enable_timing(self, on=True):
        return self._check(load().ppmlr_enable_timing(self._h, int(bool(on))))

    def read_timing(self):
        """{kind: (total_ms, launches)} for kinds x, y, z, cfl since the last read."""
        ms = (c_double * 4)()
        n = (c_longlong * 4)()
        self._check(load().ppmlr_read_timing(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(("x", "y", "z", "cfl"))}

    def set_stream(self, stream):
        return self._check(load().ppmlr_set_stream(self._h, _stream_handle(stream)))

    def autotune(self):
        ms = (c_double * 3)()
        self._check(load().ppmlr_autotune(self._h, ms))
        return list(ms)

    def tiles(self):
        C, L = (c_int * 3)(), (c_int * 3)()
        self._check(load().ppmlr_get_tiles(self._h, C, L))
        return list(C), list(L)

    def set_tiles(self, axis, C, L):
        return self._check(load().ppmlr_set_tiles(self._h, int(axis), int(C), int(L)))

    def set_march_chunk(self, axis, C):
        """Chunk length of the marching form (3) along one axis."""
        return self._check(load().ppmlr_set_march_chunk(self._h, int(axis), int(C)))

    def sweep_forms(self):
        f = (c_int * 3)()
        self._check(load().ppmlr_get_sweep_forms(self._h, f))
        return list(f)

    def set_sweep_form(self, axis, form, raise_on_error=True):
        st = load().ppmlr_set_sweep_form(self._h, int(axis), int(form))
        return self._check(st) if raise_on_error else st


def checkpoint_info(path):
    """Verify a checkpoint file on the host and return its header fields
    (raises PPMLRError for a missing, truncated or corrupt file)."""
    n, step, t, prec = (c_int * 3)(), c_longlong(), c_double(), c_int()
    st = load().ppmlr_checkpoint_info(os.fsencode(path), n, ctypes.byref(step), ctypes.byref(t), ctypes.byref(prec))
    if st != PPMLR_OK:
        raise PPMLRError(st, f"invalid checkpoint {path}")
    return {"n": list(n), "step": step.value, "time": t.value, "precision": prec.value}


class Ensemble:
    """count independent instances (own grid and boundary spec each) advanced
    together: per-instance device dt, one persistent launch per sweep, one
    CUDA graph per step."""

    def __init__(self, problems_or_specs, gamma=None, precision=PPMLR_MIXED, stream=None):
        L = load()
        items = list(problems_or_specs)
        self.count = len(items)
        self._edges, grids, bcs = [], (ppmlr_grid * self.count)(), (ppmlr_bc * self.count)()
        self.n = []
        for i, it in enumerate(items):
            edges, spec = (it.edges, it.bc) if hasattr(it, "edges") else it
            ee = [np.ascontiguousarray(e, dtype=np.float64) for e in edges]
            self._edges.append(ee)
            self.n.append(tuple(len(e) - 1 for e in ee))
            for d in range(3):
                grids[i].n[d] = self.n[i][d]
                grids[i].edges[d] = ee[d].ctypes.data_as(POINTER(c_double))
            bcs[i] = make_bc(spec)
        if gamma is None:
            gamma = items[0].gamma
        h = c_void_p()
        st = L.ppmlr_ensemble_create(self.count, grids, bcs, float(gamma), int(precision), _stream_handle(stream),
                                     ctypes.byref(h))
        if st != PPMLR_OK:
            raise PPMLRError(st, "ppmlr_ensemble_create failed")
        self._h = h
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            load().ppmlr_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != PPMLR_OK:
            raise PPMLRError(st, load().ppmlr_ensemble_last_error(self._h).decode())
        return st

    def shape(self, i):
        n = self.n[i]
        return (8, n[2], n[1], n[0])

    def set_state(self, i, U):
        if not hasattr(U, "data_ptr"):
            U = np.ascontiguousarray(U, dtype=np.float64)
        assert tuple(U.shape) == self.shape(i)
        p, dev = Context._ptrs(U)
        return self._check(load().ppmlr_ensemble_set_state(self._h, int(i), p, dev))

    def get_state(self, i, out=None):
        if out is None:
            out = np.empty(self.shape(i), dtype=np.float64)
        p, dev = Context._ptrs(out)
        self._check(load().ppmlr_ensemble_get_state(self._h, int(i), p, dev))
        return out

    def step(self, cfl, nsteps=1):
        return self._check(load().ppmlr_ensemble_step(self._h, float(cfl), int(nsteps)))

    def time_kernels(self, cfl, nsteps):
        ms = (c_double * 4)()
        self._check(load().ppmlr_ensemble_time_kernels(self._h, float(cfl), int(nsteps), ms))
        return dict(zip(("x", "y", "z", "cfl"), list(ms)))

    def autotune(self):
        ms = (c_double * 3)()
        self._check(load().ppmlr_ensemble_autotune(self._h, ms))
        return list(ms)

    def tiles(self):
        t = (c_int * 3)()
        self._check(load().ppmlr_ensemble_get_tiles(self._h, t))
        return list(t)

    def set_riemann_solver(self, iters):
        """0: two-wave Riemann solver; k > 0: k two-shock Newton steps."""
        return self._check(load().ppmlr_ensemble_set_riemann_solver(self._h, int(iters)))

    def set_steepening(self, on):
        """Contact steepening of every instance's remap (default off)."""
        return self._check(load().ppmlr_ensemble_set_steepening(self._h, int(bool(on))))

    def set_launch(self, axis, form, budget, raise_on_error=True):
        """Fix one direction's launch form (0..4) and tile budget (positions x
        lanes; + 10000 for y/z: the lanes-first tile rule)."""
        st = load().ppmlr_ensemble_set_launch(self._h, int(axis), int(form), int(budget))
        return self._check(st) if raise_on_error else st

    def dt(self):
        out = (c_double * self.count)()
        self._check(load().ppmlr_ensemble_get_dt(self._h, out))
        return list(out)

    def check(self):
        return self._check(load().ppmlr_ensemble_check(self._h))

    def diagnostics(self):
        s, f = c_longlong(), c_longlong()
        self._check(load().ppmlr_ensemble_get_diagnostics(self._h, ctypes.byref(s), ctypes.byref(f)))
        return {"step": s.value, "floor_hits": f.value}

    @property
    def launch_count(self):
        return load().ppmlr_ensemble_launch_count(self._h)
