"""Benchmark: cell-updates/s of full x/y/z steps of the split PPMLR-MHD sweep.

Default workload: the magnetosphere-shaped stretched grid 256x192x192
(x in [-100, 30] R_E, y, z in [-60, 60] R_E, finest 0.4 R_E), Earth dipole,
inner sphere r = 3 R_E, solar-wind inflow at x = +30 R_E (n = 5 cm^-3,
vx = -400 km/s, T = 1e5 K, IMF Bz = -5 nT), outflow elsewhere, FP64, CFL 0.4.
A step is the device CFL reduction plus the three sweeps; the state (604 MB)
is larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  With N > 1 (torchrun, one process per GPU)
every rank advances its own replica of the workload: the method has no
exchange step between independent domains here ("replicas only", weak
scaling), so there is no data-path collective; ranks meet only at the timing
barriers and the max-over-ranks reduction.
"""
import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per full xyz step"
UNIT = "cell-updates/s"
HBM_FALLBACK_GBS = 6800.0
# The FP64 peak of the "alu" roofline is measured in each run on the GPU in
# use (ppmlr_measure_pipe_rates: FP64 fused multiply-adds per second x 2
# flops; 503 G FMA/s = 1006 GFLOP/s on a GB300 at 2070 MHz).  The nominal
# dense FP64 rate of the part is 1.25 TFLOP/s.
FP64_NOMINAL_GFLOPS = 1250.0


def hbm_peak():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"
# Algorithmic FP64 flops (+, -, x, /, sqrt) per interior cell of one sweep on
# the magnetosphere workload (PPM coefficients counted once per zone) and per
# cell of the CFL pass, counted by the op-counting build of the oracle
# (oracle/opcount/count_flops.py, 256 x 192 x 192).
FLOPS_PER_CELL = {"x": 1189.1, "y": 1241.9, "z": 1243.7, "cfl": 207.0}
BYTES_PER_CELL_SWEEP = 128      # read 8 FP64 + write 8 FP64
# DRAM bytes per cell of one launch measured by ncu for each kernel, with the
# sha256 prefix of the kernel sources' code (comments left out) they were taken
# on (null once it changes).
# The FP64 sweeps also read the dipole table (24 B per cell) on top of the
# state: traffic above the algorithmic 128 B by that much.  The FP64 y and z
# sweeps (72-register cap) also write back their register spills: the
# blocks' dead stack frames leave L2 as DRAM writes, ~130 B per cell.  The
# FP64 CFL step's screen writes 4 B per cell that its FP64 pass reads back.
NCU_TRAFFIC = {
    "fp64:x": {"bytes_per_cell": 154.9, "src": "9ba4c5569ffc3f83"},
    "fp64:y": {"bytes_per_cell": 267.2, "src": "9ba4c5569ffc3f83"},
    "fp64:z": {"bytes_per_cell": 257.2, "src": "9ba4c5569ffc3f83"},
    # the two passes of the FP64 CFL step together (float screen 68.6, FP64 pass 4.0)
    "fp64:cfl": {"bytes_per_cell": 72.6, "src": "6549a833db154b84"},
    "mixed:x": {"bytes_per_cell": 123.6, "src": "9831875bc4f8409c"},
    "mixed:y": {"bytes_per_cell": 124.6, "src": "9831875bc4f8409c"},
    "mixed:z": {"bytes_per_cell": 124.9, "src": "9831875bc4f8409c"},
    "mixed:cfl": {"bytes_per_cell": 64.3, "src": "18b652b6cfc0a2d3"},
    # ensemble sweeps: captured on the first 8 of the 48 instances (14.9 M
    # cells; the full ensemble holds ~10 GB), scaled by cells
    "ensemble:x": {"bytes_per_cell": 125.1, "src": "be4670adf4282b76"},
    "ensemble:y": {"bytes_per_cell": 125.6, "src": "be4670adf4282b76"},
    "ensemble:z": {"bytes_per_cell": 125.5, "src": "be4670adf4282b76"},
}


# Sources of each (precision, kernel) entry of NCU_TRAFFIC; the hash of the
# files at capture time is stored with the entry.
_SWEEP = ("sweep.cuh", "launch.cuh", "march.cuh", "mixed_util.cuh", "ppmlr_internal.h")
KERNEL_SOURCES = {
    "fp64:sweep": _SWEEP + ("sweep_fp64.cu",),
    "mixed:sweep": _SWEEP + ("sweep_mixed.cu",),
    "ensemble:sweep": _SWEEP + ("sweep_mixed.cu", "ensemble.cu"),
    "fp64:cfl": ("cfl.cuh", "cfl_fp64.cu", "sweep.cuh", "mixed_util.cuh", "ppmlr_internal.h"),
    "mixed:cfl": ("cfl_mixed.cu", "cfl.cuh", "sweep.cuh", "mixed_util.cuh", "ppmlr_internal.h"),
}


def _code_only(text):
    """C/C++ source without its comments, trailing blanks and empty lines:
    what the hash of a kernel's sources covers, so that editing a comment
    does not mark a capture stale."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(key=None):
    """sha256 prefix of the code (comments left out) of the sources behind
    one NCU_TRAFFIC key ("fp64:x", "mixed:cfl", ...), or of all kernel
    sources when key is None."""
    if key is None:
        files = sorted({f for v in KERNEL_SOURCES.values() for f in v})
    else:
        prec, kern = key.split(":")
        files = KERNEL_SOURCES[f"{prec}:{'cfl' if kern == 'cfl' else 'sweep'}"]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1607_02214_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(key, cells):
    """DRAM bytes of one launch from the ncu table, or None if the kernel's
    sources changed since the capture."""
    tr = NCU_TRAFFIC.get(key)
    if tr and tr["src"] == kernel_source_hash(key):
        return tr["bytes_per_cell"] * cells
    return None


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------- ranks -------------

def max_over_ranks(x, dist=None, device="cpu"):
    """Maximum of a per-rank float over all ranks (the slowest rank sets the time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist=None, device="cpu"):
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(count, rank, world):
    """Instances of an ensemble owned by `rank`: independent problems are split
    round-robin, with no data exchanged between ranks."""
    return list(range(rank, count, world))


def throughput(cells_all_ranks, steps, max_ms):
    """Whole-job cell-updates/s: all ranks' cells x steps over the slowest rank's time."""
    return cells_all_ranks * steps / (max_ms * 1e-3)


# ---------------------------------------------------------------- clocks ------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.samples = []
        self.proc = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = ["-i", str(device_index)]
        self.cmd = ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------- workloads ------

def parse_ensemble_launch(text):
    parts = text.split(":")
    if len(parts) != 3:
        raise argparse.ArgumentTypeError("need three form,budget groups separated by ':'")
    return [tuple(int(v) for v in q.split(",")) for q in parts]


def parse_launch_config(text):
    parts = text.split(":")
    if len(parts) != 3:
        raise argparse.ArgumentTypeError("need three C,L,form groups separated by ':'")
    return [tuple(int(v) for v in q.split(",")) for q in parts]


def workload(args):
    from paper_1607_02214_gb300 import inputs
    n = tuple(args.grid)
    h0 = 0.4 * 256 / n[0] if args.h0 is None else args.h0
    prob = inputs.magnetosphere(n=n, h0=h0)
    name = f"magnetosphere_{n[0]}x{n[1]}x{n[2]}_h0_{h0:g}_{args.precision}"
    if getattr(args, "ionosphere", False):
        name += "_ionosphere"
    return prob, name


# the ionosphere shell of --ionosphere and of the bench's shell section
SHELL = dict(r_iono=1.017, r_fac=4.0, sigma_p=0.6283, n_theta=24, n_phi=48)


def config_dict(prob, name, args, world):
    d = {"workload": name, "grid": list(prob.n), "cells": prob.cells, "cfl": prob.cfl,
         "x_range_re": [-100, 30], "yz_range_re": [-60, 60], "dipole": True, "r_inner_re": 3.0,
         "inflow": "n=5 cm^-3, vx=-400 km/s, T=1e5 K, Bz=-5 nT", "precision": args.precision,
         "l2": "state 604 MB per copy > 129 MB L2: inputs larger than L2, no flush",
         "parallelism": f"replicas x{world}"}
    if getattr(args, "ionosphere", False):
        d["ionosphere_shell"] = SHELL
    return d


# ------------------------------------------------------------ reference -------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def oracle_sample(prob, steps, threads=0, keep=False):
    """Time the oracle on the host cores: `steps` steps of prob with its CFL dt.
    keep: also return the time steps and the final state."""
    import oracle
    cores = oracle.set_threads(threads)
    bc = prob.bc
    o = oracle.Oracle(prob.edges, prob.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    o.set_state(prob.U0)
    dts = []
    t0 = time.perf_counter()
    for _ in range(steps):
        dt = o.cfl_dt(prob.cfl)
        dts.append(dt)
        o.step(dt)
    t = time.perf_counter() - t0
    if keep:
        return prob.cells * steps / t, t, cores, dts, o.get_state()
    return prob.cells * steps / t, t, cores


def errors_vs(U, ref):
    """Per-variable relative L1 of U against ref, both (8, nz, ny, nx): the
    definition sum|U - ref| / sum|ref| per variable (rel_l1), the same scaled
    by each variable's group sum (rho; momentum; B'; E: rel_l1_group), and
    Linf."""
    diff = np.abs(U - ref).reshape(8, -1)
    a = np.abs(ref).reshape(8, -1).sum(axis=1)
    grp = np.array([a[0], *[a[1:4].sum()] * 3, *[a[4:7].sum()] * 3, a[7]])
    names = ["rho", "mx", "my", "mz", "Bx", "By", "Bz", "E"]
    return {"rel_l1": dict(zip(names, (diff.sum(axis=1) / np.maximum(a, 1e-300)).tolist())),
            "rel_l1_group": dict(zip(names, (diff.sum(axis=1) / grp).tolist())),
            "linf": dict(zip(names, diff.max(axis=1).tolist()))}


def run_reference(args, rank, world):
    """The oracle, as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    from paper_1607_02214_gb300 import inputs
    prob, name = workload(args)
    # one step of the full grid per timed step when it fits the time budget,
    # else the same workload at half resolution per axis (same extent)
    small = inputs.magnetosphere(n=(64, 48, 48), h0=1.6)
    rate_small, _, _ = oracle_sample(small, 1)
    est = (args.steps + args.warmup) * prob.cells / rate_small
    sample_prob, sample_desc = prob, f"one full step of {name} per timed step"
    if est > 150.0:
        n2 = tuple(max(16, k // 2) for k in prob.n)
        sample_prob = inputs.magnetosphere(n=n2, h0=0.4 * 256 / n2[0] * (prob.n[0] / 256))
        sample_desc = f"one step of the same workload at {n2[0]}x{n2[1]}x{n2[2]} per timed step"
    import oracle
    cores = oracle.set_threads(0)
    bc = sample_prob.bc
    o = oracle.Oracle(sample_prob.edges, sample_prob.gamma, bc.flat_faces(), inflow=bc.inflow,
                      dipole_moment=bc.dipole_moment, r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min,
                      powell=bc.powell)
    o.set_state(sample_prob.U0)
    for _ in range(args.warmup):
        o.step(o.cfl_dt(sample_prob.cfl))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(o.cfl_dt(sample_prob.cfl))
    t = time.perf_counter() - t0
    value = sample_prob.cells * args.steps / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_dict(prob, name, args, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return out


# ------------------------------------------------------------------ ours ------

def run_ours(args, rank, world, dist):
    import torch
    from paper_1607_02214_gb300 import build, ppmlr

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    prob, name = workload(args)
    prec = ppmlr.PPMLR_FP64 if args.precision == "fp64" else ppmlr.PPMLR_MIXED
    cells = prob.cells
    U0 = torch.from_numpy(prob.U0).cuda()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_ranks(x):
        return max_over_ranks(x, dist, "cuda")

    def timed_run(precision, steps, warmup, with_clocks=False, riemann_iters=0, steepen=False, iono=None):
        ctx = ppmlr.Context.from_problem(prob, precision)
        ctx.set_state(U0)
        ctx.set_riemann_solver(riemann_iters)
        ctx.set_steepening(steepen)
        if iono:
            ctx.set_ionosphere(**iono)
        if args.launch_config and precision == prec:
            for axis, (C, L, form) in enumerate(args.launch_config):
                if form == 3:                    # marching form: C is its chunk length
                    ctx.set_march_chunk(axis, C)
                else:
                    ctx.set_tiles(axis, C, L)
                ctx.set_sweep_form(axis, form)
        elif not args.no_autotune:
            ctx.autotune()
        ctx.step_cfl(prob.cfl, warmup)
        ctx.check()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        n0 = ctx.launch_count
        sampler = ClockSampler(local) if with_clocks else None
        if sampler:
            sampler.__enter__()
            time.sleep(0.3)
        e0.record(stream)
        for _ in range(steps):
            ctx.step_cfl(prob.cfl, 1)
        e1.record(stream)
        e1.synchronize()
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = e0.elapsed_time(e1)
        launches = ctx.launch_count - n0
        ctx.check()
        # per-kernel times in a separate pass (events between the kernels stay
        # out of the timed region above)
        ctx.enable_timing(True)
        ctx.step_cfl(prob.cfl, max(3, min(steps, 10)))
        kern = ctx.read_timing()
        ctx.enable_timing(False)
        ctx.check()
        return ctx, ms, kern, launches, (sampler.summary() if sampler else None)

    # ---- FP64 and FP32 pipe rates of this GPU (the FP64 roofline's peak)
    rates = ppmlr.measure_pipe_rates(torch.cuda.current_stream().cuda_stream)
    if args.precision == "fp64":        # the integer-pipe product beside the FP64 pipe
        rates.update(ppmlr.measure_coissue(torch.cuda.current_stream().cuda_stream))
    fp64_peak = 2.0 * rates["dfma_per_s"] * 1e-9
    hbm, hbm_src = hbm_peak()

    # ---- main measurement
    ctx, ms, kern, launches, clocks = timed_run(prec, args.steps, args.warmup, with_clocks=True,
                                                iono=SHELL if args.ionosphere else None)
    ms = max_ranks(ms)
    value = throughput(world * cells, args.steps, ms)
    log(f"[bench] {name}: {ms / args.steps:.3f} ms/step, {value:.4e} cell-updates/s, kernels {kern}")

    # ---- roofline of the dominant kernel (largest total time)
    dom = max(kern, key=lambda k: kern[k][0])
    avg_ms = kern[dom][0] / max(kern[dom][1], 1)
    src_hash = kernel_source_hash()
    traffic = ncu_traffic(f"{args.precision}:{dom}", cells)
    if args.precision == "fp64":
        ach = FLOPS_PER_CELL[dom] * cells / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "GFLOP/s",
                "frac": ach / fp64_peak, "traffic": traffic, "kernel": f"sweep_{dom}" if dom != "cfl" else "cfl",
                "avg_launch_ms": avg_ms,
                "peak_source": "measured in this run: FP64 FMA rate x 2 flops (ppmlr_measure_pipe_rates)",
                "pipe_rates": rates,
                "peak_nominal": FP64_NOMINAL_GFLOPS, "frac_of_nominal": ach / FP64_NOMINAL_GFLOPS,
                "note": "frac can exceed 1: products, reciprocals and square roots of the FP64 sweeps run "
                        "correctly rounded on the integer and FP32 pipes beside the FP64 pipe (ncu: FP64 pipe "
                        "75 % busy in x, 78 % in y)"}
    else:
        ach = BYTES_PER_CELL_SWEEP * cells / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "kernel": f"sweep_{dom}", "avg_launch_ms": avg_ms, "peak_source": hbm_src}
    # algorithmic bytes: 128 B per cell for a sweep, 64 B (the state read) for the CFL step
    per_kernel = {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1],
                      "hbm_frac_of_measured": (BYTES_PER_CELL_SWEEP if k != "cfl" else 64) * cells
                      / (v[0] / max(v[1], 1) * 1e-3) / 1e9 / hbm} for k, v in kern.items()}
    if args.precision == "fp64":
        for k, v in per_kernel.items():
            if k == "cfl":      # two passes: a float screen, FP64 only for the cells near the minimum
                v["note"] = "float screen of every cell, FP64 only for the cells near the minimum"
            else:
                v["fp64_frac_of_measured"] = FLOPS_PER_CELL[k] * cells / (v["avg_ms"] * 1e-3) / 1e9 / fp64_peak

    # ---- the other precision, and its error against the FP64 path
    extra = {}
    if not args.quick:
        other = ppmlr.PPMLR_MIXED if prec == ppmlr.PPMLR_FP64 else ppmlr.PPMLR_FP64
        octx, oms, okern, _, _ = timed_run(other, args.steps, args.warmup)
        oms = max_ranks(oms)
        ovalue = world * cells * args.steps / (oms * 1e-3)
        # accuracy: both precisions from the same state with the FP64 path's dt
        a = ppmlr.Context.from_problem(prob, ppmlr.PPMLR_FP64)
        b = ppmlr.Context.from_problem(prob, ppmlr.PPMLR_MIXED)
        a.set_state(U0)
        b.set_state(U0)
        for _ in range(args.accuracy_steps):
            dt = a.cfl_dt(prob.cfl)
            a.step(dt)
            b.step(dt)
        ua, ub = torch.empty_like(U0), torch.empty_like(U0)
        a.get_state(ua)
        b.get_state(ub)
        diff = (ub - ua).abs().reshape(8, -1)
        ref = ua.abs().reshape(8, -1).sum(dim=1)
        grp = torch.stack([ref[0], ref[1:4].sum(), ref[1:4].sum(), ref[1:4].sum(), ref[4:7].sum(), ref[4:7].sum(),
                           ref[4:7].sum(), ref[7]])
        l1 = (diff.sum(dim=1) / ref.clamp_min(1e-300)).cpu().tolist()       # per variable (the definition)
        l1g = (diff.sum(dim=1) / grp).cpu().tolist()                        # per variable, group-scaled
        linf = diff.max(dim=1).values.cpu().tolist()
        names = ["rho", "mx", "my", "mz", "Bx", "By", "Bz", "E"]
        key = "mixed" if other == ppmlr.PPMLR_MIXED else "fp64"
        odom = max(okern, key=lambda k: okern[k][0])
        oavg = okern[odom][0] / max(okern[odom][1], 1)
        obytes = (128 if odom != "cfl" else 64) * cells
        oach = obytes / (oavg * 1e-3) / 1e9
        oroof = {"bound": "hbm", "achieved": oach, "peak": hbm, "unit": "GB/s", "frac": oach / hbm,
                 "traffic": ncu_traffic(f"{key}:{odom}", cells),
                 "kernel": f"sweep_{odom}" if odom != "cfl" else "cfl", "avg_launch_ms": oavg,
                 "peak_source": hbm_src}
        extra[key] = {"value": ovalue, "ms_per_step": oms / args.steps, "roofline": oroof,
                      "tiles": {"C_L": octx.tiles(), "forms": octx.sweep_forms()},
                      "speedup_vs_fp64": (ovalue / value) if key == "mixed" else (value / ovalue),
                      "kernels_avg_ms": {k: v[0] / max(v[1], 1) for k, v in okern.items()},
                      "error_vs_fp64": {"steps": args.accuracy_steps, "rel_l1": dict(zip(names, l1)),
                                        "rel_l1_group": dict(zip(names, l1g)), "linf": dict(zip(names, linf))}}
        del a, b, octx, ua, ub

    # ---- the bit-exact FP64 form (same expression trees as the CPU reference)
    if not args.quick and args.precision == "fp64":
        xctx, xms, xkern, _, _ = timed_run(ppmlr.PPMLR_FP64_EXACT, max(3, args.steps // 2), args.warmup)
        xms = max_ranks(xms)
        nx = max(3, args.steps // 2)
        extra["fp64_exact"] = {"value": world * cells * nx / (xms * 1e-3), "ms_per_step": xms / nx,
                               "kernels_avg_ms": {k: v[0] / max(v[1], 1) for k, v in xkern.items()},
                               "note": "bit-identical to the CPU reference"}
        xctx.close()

    # ---- the nonlinear (two-shock, fast-mode) Riemann solver variant: its cost
    if not args.quick:
        nl = {"iters": 4}
        for key, p in (("fp64", ppmlr.PPMLR_FP64), ("mixed", ppmlr.PPMLR_MIXED)):
            nsteps = max(3, args.steps // 4) if key == "fp64" else args.steps
            nctx, nms, _, _, _ = timed_run(p, nsteps, args.warmup, riemann_iters=4)
            nms = max_ranks(nms)
            nl[key] = {"value": world * cells * nsteps / (nms * 1e-3), "ms_per_step": nms / nsteps}
            nctx.close()
        extra["riemann_two_shock"] = nl
        st = {}
        for key, p in (("fp64", ppmlr.PPMLR_FP64), ("mixed", ppmlr.PPMLR_MIXED)):
            nsteps = max(3, args.steps // 4) if key == "fp64" else args.steps
            sctx, sms, _, _, _ = timed_run(p, nsteps, args.warmup, steepen=True)
            sms = max_ranks(sms)
            st[key] = {"value": world * cells * nsteps / (sms * 1e-3), "ms_per_step": sms / nsteps}
            sctx.close()
        extra["contact_steepening"] = st
        if prob.bc.r_inner > 0.0 and prob.bc.dipole_moment != 0.0:
            # the ionosphere shell coupled to the inner boundary: step cost and
            # the solve alone (CUDA events around repeated solves)
            from paper_1607_02214_gb300 import inputs
            cfg = SHELL
            io = {"config": dict(cfg, sigma_p_siemens=5.0)}
            for key, p in (("fp64", ppmlr.PPMLR_FP64), ("mixed", ppmlr.PPMLR_MIXED)):
                nsteps = max(3, args.steps // 4) if key == "fp64" else args.steps
                ictx, ims, _, ilaunch, _ = timed_run(p, nsteps, args.warmup, iono=cfg)
                ims = max_ranks(ims)
                io[key] = {"value": world * cells * nsteps / (ims * 1e-3), "ms_per_step": ims / nsteps,
                           "gpu_launches_per_step": ilaunch / nsteps}
                if key == "fp64":
                    stream = torch.cuda.current_stream()
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    for _ in range(3):
                        ictx.ionosphere_solve()
                    reps = 50
                    a0.record(stream)
                    for _ in range(reps):
                        ictx.ionosphere_solve()
                    a1.record(stream)
                    a1.synchronize()
                    io["solve_ms"] = a0.elapsed_time(a1) / reps
                    phi, jr = ictx.get_ionosphere()
                    io["cross_cap_potential_kV"] = float((phi[0].max() - phi[0].min()) * inputs.V0 *
                                                         inputs.B_UNIT_NT * 1e-9 * 6.371e6 * 1e-3)
                ictx.close()
            extra["ionosphere_shell"] = io

    # ---- end to end through the C ABI with host buffers: three contexts on
    # three streams, each driven by its own host thread,
    # so that one context's host->device copy, another's device->host copy
    # and a third's kernels run at once (every step still copies its whole
    # input in from pinned host memory and its result out)
    e2e = None
    if not args.quick:
        host_in = torch.from_numpy(prob.U0).pin_memory()
        hin = host_in.numpy()
        streams = [torch.cuda.Stream() for _ in range(3)]
        ectxs = [ppmlr.Context.from_problem(prob, prec, stream=st.cuda_stream) for st in streams]
        houts = [torch.empty_like(host_in).pin_memory().numpy() for _ in ectxs]
        for c, h in zip(ectxs, houts):
            c.set_state(hin)
            c.autotune()                   # the tuned tiles (cached from the main run)
            c.step_cfl(prob.cfl, 1)
            c.get_state(h)
        per_ctx = max(1, min(args.steps, 12) // len(ectxs))
        errors = []

        def drive(c, h):
            try:
                for _ in range(per_ctx):
                    c.set_state(hin)       # host -> device, pinned; returns when copied
                    c.step_cfl(prob.cfl, 1)
                    c.get_state(h)         # device -> host; synchronises the context's stream
            except Exception as ex:        # re-raised below
                errors.append(ex)

        barrier()
        t0 = time.perf_counter()
        workers = [threading.Thread(target=drive, args=(c, h)) for c, h in zip(ectxs, houts)]
        for w in workers:
            w.start()
        for w in workers:
            w.join()
        barrier()
        t = max_ranks(time.perf_counter() - t0)
        if errors:
            raise errors[0]
        ksteps = per_ctx * len(ectxs)
        nbytes = 8 * 8 * cells
        e2e = {"value": world * cells * ksteps / t, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ksteps,
               "contexts": len(ectxs), "note": "three contexts on three streams and host threads: one step's "
                                               "input copy and another's result copy overlap a third's kernels"}
        for c in ectxs:
            c.close()
        del ectxs

    # ---- long run: graph-replayed steps, real-time factor, checkpoint I/O
    if not args.quick and not args.no_steady and world == 1:
        extra["steady"] = run_steady(args, prob, U0, barrier)

    # ---- batched ensemble: 48 seeded instances on uneven grids (mixed path);
    # with N ranks each owns a round-robin share of the instances
    if not args.quick and not args.no_ensemble:
        extra["ensemble"] = run_ensemble(args, value, barrier, rank, world, dist)

    # ---- large single domain 512x384x384 (finest 0.2 R_E), both precisions
    if not args.quick and not args.no_large and world == 1:
        extra["large"] = run_large(args, barrier, fp64_peak)

    # ---- CPU baseline: the oracle on this host's cores, bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from paper_1607_02214_gb300 import inputs
        small = inputs.magnetosphere(n=(64, 48, 48), h0=1.6)
        r_small, _, _ = oracle_sample(small, 1)
        steps = max(1, min(3, int(20.0 * r_small / cells)))
        rate, t, cores, dts, Uo = oracle_sample(prob, steps, keep=True)
        rate1, t1, _ = oracle_sample(prob, 1, threads=1)       # the same code on one core
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{steps} full step(s) of {name}, OpenMP over pencils, {t:.1f} s",
               "single_core": {"value": rate1, "sample": f"1 full step on 1 thread, {t1:.1f} s"},
               "cpu_model": cpu_model()}
        # the GPU paths replayed with the oracle's time steps: their error
        # against the oracle on the full workload
        acc = {"steps": steps}
        for key, p in (("fp64", ppmlr.PPMLR_FP64), ("mixed", ppmlr.PPMLR_MIXED)):
            c = ppmlr.Context.from_problem(prob, p)
            c.set_state(U0)
            for dt in dts:
                c.step(dt)
            c.check()
            acc[key] = errors_vs(c.get_state(), Uo)
            c.close()
        extra["error_vs_oracle"] = acc
        del Uo

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(prob, name, args, world), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
           "clocks": clocks, "gpu_launches": launches, "kernels": per_kernel, "kernel_src": src_hash,
           "tiles": {"C_L": ctx.tiles(), "forms": ctx.sweep_forms()}}
    out.update(extra)
    return out


def run_steady(args, prob, U0, barrier):
    """The magnetosphere run as it is used in production: many steps with the
    device CFL time step, replayed from CUDA graphs of 16 steps.  Reports the
    real-time factor (simulated seconds per wall-clock second; the code time
    unit is R_E / 100 km/s) per precision, and the time to write and read a
    checksummed checkpoint of the state."""
    import tempfile
    import torch
    from paper_1607_02214_gb300 import inputs, ppmlr
    t_unit = inputs.R_E_KM * 1e3 / inputs.V0
    out = {"graph_steps": 16, "time_unit_s": t_unit}
    for key, precision, nsteps in (("mixed", ppmlr.PPMLR_MIXED, 640), ("fp64", ppmlr.PPMLR_FP64, 48)):
        ctx = ppmlr.Context.from_problem(prob, precision)
        ctx.set_state(U0)
        ctx.autotune()
        ctx.run(prob.cfl, 16, graph_steps=16)      # captures both parities' graphs
        ctx.run(prob.cfl, 16, graph_steps=16)
        ctx.check()
        t_start = ctx.time
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        ctx.run(prob.cfl, nsteps, graph_steps=16)
        e1.record(stream)
        e1.synchronize()
        wall = e0.elapsed_time(e1) * 1e-3
        ctx.check()
        sim = (ctx.time - t_start) * t_unit
        out[key] = {"steps": nsteps, "ms_per_step": wall * 1e3 / nsteps, "sim_seconds": sim, "wall_seconds": wall,
                    "real_time_factor": sim / wall, "mean_dt_s": sim / nsteps}
        if key == "mixed":
            with tempfile.TemporaryDirectory() as d:
                path = os.path.join(d, "state.ck")
                t0 = time.perf_counter()
                ctx.checkpoint_save(path)
                t1 = time.perf_counter()
                ctx.checkpoint_load(path)
                t2 = time.perf_counter()
                size = os.path.getsize(path)
            out["checkpoint"] = {"bytes": size, "save_s": t1 - t0, "load_s": t2 - t1}
        ctx.close()
    log(f"[bench] steady: real-time factor mixed {out['mixed']['real_time_factor']:.1f}, "
        f"fp64 {out['fp64']['real_time_factor']:.2f}")
    return out


def run_ensemble(args, fp64_value, barrier, rank=0, world=1, dist=None):
    """48 magnetosphere instances, grids drawn from {96^3, 128x96x96, 160x128x128},
    seeded solar wind; one launch per sweep over all instances, one CUDA graph
    per step.  With N ranks, rank r advances instances r, r+N, ... (no data
    exchanged; the whole job's throughput is reported)."""
    import torch
    from paper_1607_02214_gb300 import inputs, ppmlr
    t0 = time.perf_counter()
    all_probs = inputs.ensemble(48)[:args.ensemble_count]
    probs = [all_probs[i] for i in shard(len(all_probs), rank, world)]
    log(f"[bench] ensemble inputs built in {time.perf_counter() - t0:.1f} s")
    cells = sum(p.cells for p in probs)
    cells_all = sum(p.cells for p in all_probs)
    out = {"workload": f"ensemble_{len(all_probs)}_magnetosphere_mixed", "instances": len(all_probs),
           "cells": cells_all,
           "grids": sorted({"x".join(map(str, p.n)) for p in all_probs}),
           "scaling": "strong" if world > 1 else None, "instances_per_rank": len(probs)}
    ens = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_MIXED)
    for i, p in enumerate(probs):
        ens.set_state(i, p.U0)
    if args.ensemble_launch:
        for axis, (form, budget) in enumerate(args.ensemble_launch):
            ens.set_launch(axis, form, budget)
    else:
        out["tuned_ms"] = ens.autotune()
    out["tile_thread_budget"] = ens.tiles()
    ens.step(0.4, args.warmup)
    ens.check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    n0 = ens.launch_count
    e0.record(stream)
    ens.step(0.4, args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ens.check()
    out.update({"value": throughput(cells_all, args.steps, ms), "unit": UNIT, "ms_per_step": ms / args.steps,
                "gpu_launches": ens.launch_count - n0, "graph_replay": True})
    out["speedup_vs_fp64"] = out["value"] / fp64_value if fp64_value and np.isfinite(fp64_value) else None
    if world > 1:        # the per-kernel and comparison runs below are single-GPU diagnostics
        ens.close()
        return out
    kern = ens.time_kernels(0.4, 3)
    out["kernels_avg_ms"] = kern
    dom = max(("x", "y", "z"), key=lambda k: kern[k])
    ach = BYTES_PER_CELL_SWEEP * cells / (kern[dom] * 1e-3) / 1e9
    hbm, hbm_src = hbm_peak()
    out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                       "traffic": ncu_traffic(f"ensemble:{dom}", cells),
                       "kernel": f"sweep_ensemble_{dom}", "avg_launch_ms": kern[dom], "peak_source": hbm_src}
    # the same instances advanced one context at a time (no batching)
    ctxs = [ppmlr.Context.from_problem(p, ppmlr.PPMLR_MIXED) for p in probs]
    for c, p in zip(ctxs, probs):
        c.set_state(p.U0)
        c.step_cfl(0.4, 1)
    barrier()
    e0.record(stream)
    for _ in range(3):
        for c in ctxs:
            c.step_cfl(0.4, 1)
    e1.record(stream)
    e1.synchronize()
    out["loop_of_contexts_value"] = cells * 3 / (e0.elapsed_time(e1) * 1e-3)
    out["speedup_vs_loop_of_contexts"] = out["value"] / out["loop_of_contexts_value"]
    for c in ctxs:
        c.close()
    del ctxs
    # error against the FP64 ensemble (each with its own device dt)
    nerr = 10
    a = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_FP64)
    b = ppmlr.Ensemble(probs, precision=ppmlr.PPMLR_MIXED)
    for i, p in enumerate(probs):
        a.set_state(i, p.U0)
        b.set_state(i, p.U0)
    a.step(0.4, nerr)
    b.step(0.4, nerr)
    worst, worst_g = 0.0, 0.0
    for i in range(len(probs)):
        ua, ub = a.get_state(i), b.get_state(i)
        ref = np.abs(ua).reshape(8, -1).sum(axis=1)
        grp = np.array([ref[0], *[ref[1:4].sum()] * 3, *[ref[4:7].sum()] * 3, ref[7]])
        d = np.abs(ub - ua).reshape(8, -1).sum(axis=1)
        worst = max(worst, float((d / np.maximum(ref, 1e-300)).max()))
        worst_g = max(worst_g, float((d / grp).max()))
    out["error_vs_fp64"] = {"steps": nerr, "max_rel_l1_over_instances_and_variables": worst,
                            "max_rel_l1_group_over_instances_and_variables": worst_g}
    a.close()
    b.close()
    ens.close()
    return out


def run_large(args, barrier, fp64_peak):
    """512x384x384 stretched grid (finest 0.2 R_E), same extent and boundaries."""
    import torch
    from paper_1607_02214_gb300 import inputs, ppmlr
    prob = inputs.magnetosphere(n=(512, 384, 384), h0=0.2)
    cells = prob.cells
    out = {"workload": "magnetosphere_512x384x384_h0_0.2", "cells": cells}
    U0 = torch.from_numpy(prob.U0).cuda()
    for name, prec, steps in (("fp64", ppmlr.PPMLR_FP64, 5), ("mixed", ppmlr.PPMLR_MIXED, 20)):
        ctx = ppmlr.Context.from_problem(prob, prec)
        ctx.set_state(U0)
        ctx.autotune()
        ctx.step_cfl(prob.cfl, 3)
        ctx.check()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        ctx.step_cfl(prob.cfl, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ctx.check()
        ctx.enable_timing(True)                 # per-kernel times: a separate pass
        ctx.step_cfl(prob.cfl, max(3, min(steps, 6)))
        kern = ctx.read_timing()
        ctx.enable_timing(False)
        ctx.check()
        hbm, _ = hbm_peak()
        per = {}
        for k, (tot, n) in kern.items():
            avg = tot / max(n, 1)
            byts = (BYTES_PER_CELL_SWEEP if k != "cfl" else 64) * cells
            per[k] = {"avg_ms": avg, "hbm_frac_of_measured": byts / (avg * 1e-3) / 1e9 / hbm}
            if name == "fp64" and k != "cfl":     # (the FP64 CFL step is a float screen plus a few cells)
                per[k]["fp64_gflops"] = FLOPS_PER_CELL[k] * cells / (avg * 1e-3) / 1e9
                per[k]["fp64_frac_of_measured"] = per[k]["fp64_gflops"] / fp64_peak
        out[name] = {"value": cells * steps / (ms * 1e-3), "ms_per_step": ms / steps, "steps": steps,
                     "kernels": per, "tiles": ctx.tiles(), "forms": ctx.sweep_forms()}
        ctx.close()
    out["mixed"]["speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    del U0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--grid", type=int, nargs=3, default=[256, 192, 192])
    ap.add_argument("--h0", type=float, default=None)
    ap.add_argument("--accuracy-steps", type=int, default=50)
    ap.add_argument("--quick", action="store_true", help="main measurement only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-steady", action="store_true", help="skip the long graph-replayed run")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--ionosphere", action="store_true",
                    help="main measurement with the ionosphere shell coupled to the inner boundary")
    ap.add_argument("--launch-config", type=parse_launch_config, default=None,
                    help="fixed tiles and launch forms of the main precision instead of the autotuner: "
                         "C,L,form for x:y:z, e.g. 256,1,0:64,4,2:64,4,2")
    ap.add_argument("--ensemble-only", action="store_true", help="only the 48-instance ensemble section")
    ap.add_argument("--ensemble-count", type=int, default=48,
                    help="the first N of the 48 seeded ensemble instances (smaller captures)")
    ap.add_argument("--ensemble-launch", type=parse_ensemble_launch, default=None,
                    help="fixed ensemble launch form,budget per direction (x:y:z) instead of the autotuner; "
                         "budget + 10000 = lanes-first tiles (y, z)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("[bench] warm-up raised to 3 steps")
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend)
        dist = tdist

    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.ensemble_only:
        import torch
        from paper_1607_02214_gb300 import build
        build.build()
        out = run_ensemble(args, float("nan"), torch.cuda.synchronize)
    else:
        out = run_ours(args, rank, world, dist)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
