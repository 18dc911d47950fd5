"""Block decomposition along z (paper_1607_02214_gb300/decomp.py) on the CPU:
slab geometry, and whole runs split over 2 and 3 ranks -- in one process and
as gloo process groups -- against the single-domain oracle, bit for bit
(owned cells see exactly the single domain's arithmetic), with identical
CFL time steps.  The engine of each slab is the oracle itself behind the
library's method names (sweep, cfl_dt, get_layers, set_layers)."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1607_02214_gb300 import decomp, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEPS = 4                     # both step parities, each with its exchange


class OracleEngine:
    """A slab's problem run by the oracle, with the library's methods."""

    def __init__(self, prob):
        bc = prob.bc
        self.o = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow,
                               dipole_moment=bc.dipole_moment, r_inner=bc.r_inner, inner=bc.inner,
                               p_min=bc.p_min, powell=bc.powell)
        self.o.set_state(prob.U0)

    def sweep(self, axis, dt):
        assert self.o.sweep(axis, dt) == 0

    def cfl_dt(self, cfl):
        return self.o.cfl_dt(cfl)

    def get_layers(self, k0, nk, out=None):
        data = self.o.get_state()[:, k0:k0 + nk]
        if out is None:
            return data.copy()
        out[...] = data if isinstance(out, np.ndarray) else __import__("torch").from_numpy(data)
        return out

    def set_layers(self, k0, U):
        U = U.numpy() if hasattr(U, "numpy") else U
        S = self.o.get_state()
        S[:, k0:k0 + U.shape[1]] = U
        self.o.set_state(S)

    def get_state(self):
        return self.o.get_state()


def magnetosphere():
    return inputs.magnetosphere(n=(24, 20, 24), h0=2.0, x_ext=(-30, 20), yz_ext=(-25, 25))


def periodic_dyadic():
    # edges k/32 (exactly representable, so the wrapped halo images have the
    # single domain's widths bit for bit)
    n = (16, 12, 32)
    edges = [np.arange(k + 1) / 32.0 for k in n]
    U = inputs.random_smooth_state(n, 17, edges=edges)
    return inputs.Problem("periodic", edges, 5.0 / 3.0, inputs.BoundarySpec(powell=1), U)


def single_domain(prob):
    e = OracleEngine(prob)
    dts = []
    for _ in range(NSTEPS):
        dt = e.cfl_dt(prob.cfl)
        dts.append(dt)
        assert e.o.step(dt) == 0
    return e.get_state(), dts


def test_slab_geometry():
    s = decomp.slabs(40, 3, periodic=False)
    assert [(x.z0, x.z1) for x in s] == [(0, 13), (13, 26), (26, 40)]
    assert [(x.hlo, x.hhi) for x in s] == [(0, 7), (7, 7), (7, 0)]
    assert [(x.lo_nb, x.hi_nb) for x in s] == [(None, 1), (0, 2), (1, None)]
    p = decomp.slabs(32, 2, periodic=True)
    assert [(x.lo_nb, x.hi_nb, x.hlo, x.hhi) for x in p] == [(1, 1, 7, 7), (0, 0, 7, 7)]
    assert decomp.slabs(5, 1, periodic=True)[0] == decomp.Slab(0, 0, 5, 0, 0, None, None)
    with pytest.raises(ValueError):
        decomp.slabs(20, 3, periodic=False)        # fewer than 7 layers per rank


def test_local_problems_are_slices_of_the_global_one():
    pr = periodic_dyadic()
    w = np.diff(pr.edges[2])
    for s in decomp.slabs(32, 3, periodic=True):
        lp = decomp.local_problem(pr, s)
        gz = np.mod(np.arange(s.z0 - s.hlo, s.z1 + s.hhi), 32)
        assert np.array_equal(np.diff(lp.edges[2]), w[gz])             # widths bit for bit, wrapped
        assert np.array_equal(lp.U0, pr.U0[:, gz])
        assert lp.bc.face[2] == (inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    m = magnetosphere()
    s0 = decomp.slabs(24, 2, periodic=False)[0]
    lp = decomp.local_problem(m, s0)
    assert np.array_equal(lp.edges[2], m.edges[2][:s0.z1 + 7 + 1])
    assert lp.bc.face[2] == (m.bc.face[2][0], inputs.BC_OUTFLOW)


@pytest.mark.parametrize("case,world", [("magnetosphere", 2), ("magnetosphere", 3), ("periodic", 2),
                                        ("periodic", 3)])
def test_split_run_in_one_process_is_bit_identical(case, world):
    pr = magnetosphere() if case == "magnetosphere" else periodic_dyadic()
    ref, dts = single_domain(pr)
    run = decomp.ZSlabRun(pr, world, list(range(world)), OracleEngine, decomp.LocalTransport())
    got_dts = []
    for _ in range(NSTEPS):
        dt = run.cfl_dt(pr.cfl)
        got_dts.append(dt)
        run.step(dt)
    assert got_dts == dts
    U = np.concatenate([run.owned_state(i) for i in range(world)], axis=1)
    assert np.array_equal(U, ref)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def gloo_worker(rank, world, port, case, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    import torch.distributed as dist

    from test_decomp import OracleEngine, magnetosphere, periodic_dyadic
    from paper_1607_02214_gb300 import decomp as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = magnetosphere() if case == "magnetosphere" else periodic_dyadic()
    run = D.ZSlabRun(pr, world, [rank], OracleEngine, D.DistTransport(dist))
    dts = []
    for _ in range(NSTEPS):
        dt = run.cfl_dt(pr.cfl)
        dts.append(dt)
        run.step(dt)
    np.save(os.path.join(out_dir, f"u{rank}.npy"), run.owned_state())
    np.save(os.path.join(out_dir, f"dt{rank}.npy"), np.array(dts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("magnetosphere", 2), ("periodic", 2), ("periodic", 3)])
def test_split_run_over_gloo_ranks_is_bit_identical(case, world, tmp_path):
    import torch.multiprocessing as mp
    pr = magnetosphere() if case == "magnetosphere" else periodic_dyadic()
    ref, dts = single_domain(pr)
    mp.spawn(gloo_worker, args=(world, free_port(), case, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert np.load(tmp_path / f"dt{r}.npy").tolist() == dts
    U = np.concatenate([np.load(tmp_path / f"u{r}.npy") for r in range(world)], axis=1)
    assert np.array_equal(U, ref)
