"""The allocation-free CFL entry point (ppmlr_cfl_dt_noalloc).

It serves callers that may not allocate device memory: they pass the state,
the grid geometry and the output as their own device arrays, and the call
uses only a static scratch array inside the library.  This test calls it
through the C ABI twice in a row and checks each result against the
context-based ppmlr_cfl_dt on the same state (default FP64 context: within
1e-11; exact-form context: bit for bit) and against the CPU reference's CFL
time step (bit for bit: the same IEEE double sequence).  It lives in its own
file that pytest collects last, and it passes both alone in a fresh process
and after the other tests (the static scratch keeps the previous call's
contents, so the second call also checks that the entry point clears what
must start at zero).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_cfl_matches_context_cfl_twice():
    import torch

    import oracle
    from paper_1607_02214_gb300 import build, inputs, ppmlr
    build.build()
    L = ppmlr.load()
    prob = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    ctx = ppmlr.Context.from_problem(prob, ppmlr.PPMLR_FP64)
    U = torch.from_numpy(prob.U0).cuda()
    ctx.set_state(U)
    exact = ppmlr.Context.from_problem(prob, ppmlr.PPMLR_FP64_EXACT)
    bc = prob.bc
    orc = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                        r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)

    geo = []
    for e in prob.edges:
        w = torch.from_numpy(e[1:] - e[:-1]).cuda()
        c = torch.from_numpy(0.5 * (e[:-1] + e[1:])).cuda()
        geo.append((w, c))
    n = (ctypes.c_int * 3)(*prob.n)
    wp = (ctypes.POINTER(ctypes.c_double) * 3)(*[ctypes.cast(g[0].data_ptr(), ctypes.POINTER(ctypes.c_double))
                                                 for g in geo])
    cp = (ctypes.POINTER(ctypes.c_double) * 3)(*[ctypes.cast(g[1].data_ptr(), ctypes.POINTER(ctypes.c_double))
                                                 for g in geo])
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def noalloc(state):
        ptrs, _ = ppmlr.Context._ptrs(state)
        st = L.ppmlr_cfl_dt_noalloc(ptrs, n, wp, cp, prob.gamma, bc.p_min, bc.dipole_moment, bc.r_inner,
                                    prob.cfl, 0, ctypes.cast(dt_dev.data_ptr(), ctypes.POINTER(ctypes.c_double)),
                                    stream)
        assert st == ppmlr.PPMLR_OK
        torch.cuda.synchronize()
        return float(dt_dev.item())

    for call in range(2):
        ref = ctx.cfl_dt(prob.cfl)                    # existing entry point
        state = torch.empty_like(U)
        ctx.get_state(state)
        got = noalloc(state)                          # allocation-free entry point
        assert np.isfinite(got) and got > 0
        assert abs(got - ref) <= 1e-11 * abs(ref), (call, got, ref)
        exact.set_state(state)
        assert got == exact.cfl_dt(prob.cfl), call    # exact-form context: bit for bit
        orc.set_state(state.cpu().numpy())
        assert got == orc.cfl_dt(prob.cfl), call      # CPU reference: bit for bit
        ctx.step(ref)                                 # a different state for the second call

    # sizes beyond the static scratch are rejected
    ptrs, _ = ppmlr.Context._ptrs(U)
    st = L.ppmlr_cfl_dt_noalloc(ptrs, n, wp, cp, prob.gamma, bc.p_min, bc.dipole_moment, bc.r_inner, prob.cfl,
                                4096, ctypes.cast(dt_dev.data_ptr(), ctypes.POINTER(ctypes.c_double)), stream)
    assert st == ppmlr.PPMLR_E_INVALID
