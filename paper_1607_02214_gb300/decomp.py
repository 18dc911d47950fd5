"""One domain split along z across ranks: block decomposition with a halo
exchange (the paper's own scaling axis: MPI subdomains exchanging boundary
data, Secs. III-A and III-B).

GB300 form: one process per GPU.  Rank r owns the z layers [z0, z1) of the
global grid; its context (the ordinary single-domain library) holds that slab
plus GH = 7 halo layers (the stencil radius of one sweep) toward each
neighbour.  The x and y sweeps are complete pencils inside every slab, so
they need no data from other ranks and keep valid halos valid; a z sweep
leaves its halo layers stale (their stencils reach past the slab), so the
halos are refreshed from the neighbours' owned layers right after every z
sweep: one exchange per step, GH layers x 8 arrays per face.  The CFL time
step is the minimum over the ranks (all-reduce min): every rank's local
minimum runs over owned and halo cells, all of them cells of the global grid
with current values, so the minimum over ranks is the global one.  Owned
cells thus see exactly the arithmetic of the single domain; the exact FP64
form reproduces the single-domain run bit for bit.  A slab face that borders
another rank is given an outflow face in its local context: its ghosts only
reach the halo layers, never an owned cell.

The exchange goes through a transport: `DistTransport` (torch.distributed,
point-to-point sends of the halo blocks -- NCCL between GPUs, gloo on CPU;
the received layers are copied into the local state, no kernel reads a
peer's memory) or `LocalTransport` (every slab in one process, direct
copies: tests).  The engine of a slab is any object with the single-domain
methods `sweep(axis, dt)`, `cfl_dt(cfl)`, `get_layers(k0, nk, out)`,
`set_layers(k0, U)` and `get_state()`, such as `ppmlr.Context`.
"""
import dataclasses
from typing import List, Optional

import numpy as np

from . import inputs

GH = 7


@dataclasses.dataclass
class Slab:
    rank: int
    z0: int                    # owned global layers [z0, z1)
    z1: int
    hlo: int                   # halo layers below / above the owned ones (0 or GH)
    hhi: int
    lo_nb: Optional[int]       # neighbour rank below / above (None at a physical face)
    hi_nb: Optional[int]

    @property
    def nown(self) -> int:
        return self.z1 - self.z0

    @property
    def nlocal(self) -> int:
        return self.hlo + self.nown + self.hhi


def slabs(nz: int, world: int, periodic: bool) -> List[Slab]:
    """Nearly equal owned ranges of the nz layers; every rank owns at least GH
    layers so that a halo comes from one neighbour only."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if world == 1:
        return [Slab(0, 0, nz, 0, 0, None, None)]
    if nz < GH * world:
        raise ValueError(f"{nz} layers cannot give {world} ranks {GH} layers each")
    bounds = [nz * r // world for r in range(world + 1)]
    out = []
    for r in range(world):
        lo = r - 1 if r > 0 else (world - 1 if periodic else None)
        hi = r + 1 if r < world - 1 else (0 if periodic else None)
        out.append(Slab(r, bounds[r], bounds[r + 1], GH if lo is not None else 0, GH if hi is not None else 0,
                        lo, hi))
    return out


def local_problem(prob: "inputs.Problem", s: Slab) -> "inputs.Problem":
    """The slab's own problem: owned layers plus halos (global cells, wrapped
    across a periodic z axis), faces bordering another rank made outflow."""
    ez = np.asarray(prob.edges[2], dtype=np.float64)
    nz = len(ez) - 1
    lo, hi = s.z0 - s.hlo, s.z1 + s.hhi
    if lo >= 0 and hi <= nz:
        ez_loc = ez[lo:hi + 1].copy()              # a slice of the global edges: identical widths and centres
    else:                                          # periodic wrap: the neighbouring images of the far cells
        L = ez[nz] - ez[0]
        idx = np.arange(lo, hi + 1)
        ez_loc = ez[np.mod(idx, nz)] + L * np.floor_divide(idx, nz)
        ez_loc[idx == nz] = ez[nz]
    gz = np.mod(np.arange(lo, hi), nz)
    U0 = np.ascontiguousarray(np.take(prob.U0, gz, axis=1))
    face = [list(f) for f in prob.bc.face]
    if s.hlo:
        face[2][0] = inputs.BC_OUTFLOW             # its ghosts reach only the halo layers
    if s.hhi:
        face[2][1] = inputs.BC_OUTFLOW
    bc = dataclasses.replace(prob.bc, face=tuple(tuple(f) for f in face))
    return inputs.Problem(f"{prob.name}_z{s.rank}", [prob.edges[0], prob.edges[1], ez_loc], prob.gamma, bc, U0,
                          prob.cfl)


class ZSlabRun:
    """Advances a domain split along z: the library's step (x, y, z sweeps
    on even steps, z, y, x on odd ones) on every slab held here, halos
    refreshed after each z sweep, the CFL step the minimum over all ranks.

    prob: the global problem; world: number of ranks; ranks: the ranks whose
    slabs this process holds (one with DistTransport, all with
    LocalTransport); make_engine(local_problem) -> engine with the slab's
    initial state set."""

    def __init__(self, prob, world, ranks, make_engine, transport):
        nz = prob.n[2]
        periodic = prob.bc.face[2][0] == inputs.BC_PERIODIC
        self.world = world
        self.all_slabs = slabs(nz, world, periodic)
        self.slabs = [self.all_slabs[r] for r in ranks]
        self.engines = [make_engine(local_problem(prob, s)) for s in self.slabs]
        self.transport = transport
        self.plane = (prob.n[1], prob.n[0])
        self.steps = 0

    def cfl_dt(self, cfl: float) -> float:
        return self.transport.min_all(min(e.cfl_dt(cfl) for e in self.engines))

    def step(self, dt: float) -> None:
        for axis in ((0, 1, 2) if self.steps % 2 == 0 else (2, 1, 0)):
            for e in self.engines:
                e.sweep(axis, dt)
            if axis == 2 and self.world > 1:
                self.exchange()
        self.steps += 1

    def exchange(self) -> None:
        sends = []
        for s, e in zip(self.slabs, self.engines):
            lo = e.get_layers(s.hlo, GH, out=self.transport.empty((8, GH) + self.plane)) \
                if s.lo_nb is not None else None
            hi = e.get_layers(s.hlo + s.nown - GH, GH, out=self.transport.empty((8, GH) + self.plane)) \
                if s.hi_nb is not None else None
            sends.append((s, lo, hi))
        for (s, _, _), e, (rlo, rhi) in zip(sends, self.engines, self.transport.exchange(sends)):
            if rlo is not None:
                e.set_layers(0, rlo)
            if rhi is not None:
                e.set_layers(s.hlo + s.nown, rhi)

    def owned_state(self, i: int = 0):
        """The owned layers of the i-th slab held here, (8, nown, ny, nx)."""
        s = self.slabs[i]
        return self.engines[i].get_layers(s.hlo, s.nown)


class LocalTransport:
    """Every slab in this process: the halos are copied directly (tests)."""

    def empty(self, shape):
        return np.empty(shape, dtype=np.float64)

    def min_all(self, x: float) -> float:
        return float(x)

    def exchange(self, sends):
        by_rank = {s.rank: (lo, hi) for s, lo, hi in sends}
        out = []
        for s, _, _ in sends:
            rlo = by_rank[s.lo_nb][1] if s.lo_nb is not None else None   # the lower neighbour's top owned layers
            rhi = by_rank[s.hi_nb][0] if s.hi_nb is not None else None   # the upper neighbour's bottom owned layers
            out.append((rlo, rhi))
        return out


class DistTransport:
    """One slab per process, torch.distributed point-to-point sends (NCCL
    between GPUs, gloo on CPU).  Two phases, each a matched pair of one send
    and one receive per rank: up (own top layers to the upper neighbour, the
    lower neighbour's into the bottom halo), then down; the pairing holds
    under in-order matching too, including two ranks on a periodic axis."""

    def __init__(self, dist, device=None, group=None):
        self.dist, self.device, self.group = dist, device, group

    def empty(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    def _t(self, x):
        import torch
        return x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))

    def min_all(self, x: float) -> float:
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return float(t.item())

    def exchange(self, sends):
        (s, lo, hi), = sends
        rlo = rhi = None
        # phase 1 (up): top owned layers -> upper neighbour; bottom halo <- lower neighbour
        reqs = []
        if s.hi_nb is not None:
            reqs.append(self.dist.isend(self._t(hi), s.hi_nb, group=self.group, tag=1))
        if s.lo_nb is not None:
            rlo = self.empty(tuple(lo.shape))
            reqs.append(self.dist.irecv(rlo, s.lo_nb, group=self.group, tag=1))
        for r in reqs:
            r.wait()
        # phase 2 (down): bottom owned layers -> lower neighbour; top halo <- upper neighbour
        reqs = []
        if s.lo_nb is not None:
            reqs.append(self.dist.isend(self._t(lo), s.lo_nb, group=self.group, tag=2))
        if s.hi_nb is not None:
            rhi = self.empty(tuple(hi.shape))
            reqs.append(self.dist.irecv(rhi, s.hi_nb, group=self.group, tag=2))
        for r in reqs:
            r.wait()
        return [(rlo, rhi)]
