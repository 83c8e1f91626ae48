"""Benchmark of the SMC hot path on GB300.

A step is one time step of the configured integrator over the whole box
array (every kernel of the path: ghost gather, primitives and transport,
velocity gradients, the three stencil directions, correction-velocity and
reaction terms, the SDC node updates or the multirate fine-node chains).

Default workload ``c4``: 64 boxes of 16..64 cells per edge tiling a periodic
domain, 21 species / 84 reactions, multirate SDC with 3 coarse
(advection-diffusion) and 5 fine (reaction) Gauss-Lobatto nodes, 4 sweeps.

value = cells x advection-diffusion RHS evaluations per step / time (Mcell-RHS/s),
with K M1 = 8 such evaluations per multirate step after the first (the
first value f(U_0) is recycled, Sec. 3.1); the K M2 reaction evaluations of
the fine nodes are part of the step's time.  The headline is the FP64 path
(the paper's precision); the mixed FP32/FP64 path and its error are reported
beside it under "precisions".

Arithmetic rooflines divide by FMA-pipe throughputs measured on the same GPU
in the same run (smc_fma_throughput), HBM ones by the measured copy
bandwidth of MEASURED_PEAKS.json.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl smc|reference]
                       [--workload c1|c2|c3|c4|c5|t1|t2|peaks] [--precision fp64]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smc", choices=["smc", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--precision", default="both",
                    choices=["fp64", "mixed", "mixed_rates32", "both", "fp64+mixed"],
                    help="both: FP64 is the headline, mixed and mixed with FP32-mantissa rates "
                         "measured beside it; fp64+mixed: the first two only")
    ap.add_argument("--lean", action="store_true",
                    help="skip the kernel-by-kernel (no graph) timing pass (long-step workloads)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--n", type=int, default=None,
                    help="smaller instance of the workload (profiling captures)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--tiles", default=None,
                    help="segment,x_layout,march[,persistent]: use this stencil schedule instead "
                         "of autotuning")
    ap.add_argument("--fine-repeat", type=int, default=1,
                    help="multirate fine-node groups per coarse interval (1: type (b), >1: type (c))")
    ap.add_argument("--sdc-exit", type=float, default=0.0,
                    help="residual early-exit threshold (0: every sweep runs)")
    ap.add_argument("--mr-mode", type=int, default=1, choices=(1, 2),
                    help="multirate mode: 1 explicit reactions on the fine nodes, 2 implicit "
                         "reactions (BDF) on the coarse nodes, advection-diffusion on the fine")
    return ap.parse_args()


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def job_throughput(world, ncells, evals_per_step, ms_per_step):
    """Whole-job Mcell-RHS/s: every rank advances its own replica of the
    workload, so the job processes world x ncells x evals cells per step in
    the slowest rank's step time."""
    return world * ncells * evals_per_step / (ms_per_step / 1e3) / 1e6


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def march_flops_per_cell(ns: int, mode: int = 0) -> float:
    """FP64 flops one stencil-direction kernel (k_march) spends per cell,
    counted from its source (an FMA is 2 flops): narrow-stencil face fluxes
    490 + 134 ns (difference-first: 87 per M u, 81 per M^T a, 20 per
    difference dot, 15 per plain dot), flux differences 4 + 2 ns, convective
    + mixed viscous D 225 + 21 ns, correction velocity 27 + 28 ns,
    accumulation 5 + ns."""
    vc = 27 + 28 * ns if mode == 0 else 0
    return 490 + 134 * ns + 4 + 2 * ns + 225 + 21 * ns + vc + 5 + ns


def march_flops_per_cell_mixed(ns: int, mode: int = 0) -> float:
    """FP32 flops of the mixed-precision stencil-direction kernel per cell,
    counted from its source like march_flops_per_cell, with the float-pair
    work: each pair difference costs 3 flops, each pair product 7."""
    # faces: M u on pairs (44 fma + 7 pair diffs) = 109, M^T a = 81, pair dot
    # (7 fma + 7 pair diffs) = 35, plain dot = 15
    face = 109 + 2 * 81 + 3 * 35 + 3 * 35 + 2 + (109 + 15 + 1) + 16 + ns * (109 + 3 * 15 + 2)
    diffs = 4 + 2 * ns
    conv = 8 * (5 * 7 + 12) + 4 * (5 * 5 + 3 * 3) + 5 + ns * (4 * (2 * 7 + 3 + 2) + 1)
    vc = (4 * 5 + 2) + ns * (4 * 5 + 2) + ns * (4 * 5 + 2) + (4 * 5 + 2) if mode == 0 else 0
    return face + diffs + conv + vc + 5 + ns


EXP_FLOPS = 14.0      # FP64 flops of one table-driven exponential in FP64 arithmetic


def chem_flops_per_eval(ns: int, nr: int, alu: int = 1) -> float:
    """FP64 flops of one reaction-term evaluation per cell (FMA = 2), counted
    from the source: per reaction 34 (exponent 7.6, concentration products
    2.5, table-driven exponential 14, net rate 3, species updates 7.2), per
    species 43 (Gibbs energy 12, shift 2, z_k with its exponential 15,
    mixture polynomial of the Newton solve 14), per cell 210 (ln T, 1/T,
    the pressure powers with their exponential, 1/rho, velocities, the
    Newton iterations).  Cross-checked with ncu's DFMA/DMUL/DADD counts of
    k_fine_chain (4132 per evaluation at 21 species / 84 reactions against
    3969 counted).  alu >= 1 (SMC_OPT_ALU, the default): the exponentials,
    one per reaction, per species and per cell, run on the integer and FP32
    pipes, and the count is that of the FP64 pipe (14 flops less each)."""
    flops = 34.0 * nr + 43.0 * ns + 210.0
    if alu:
        flops -= EXP_FLOPS * (nr + ns + 1)
    return flops


def chem_flops_per_eval_rates32(ns: int, nr: int) -> float:
    """FP64 flops of the same evaluation with FP32-mantissa rates: per
    reaction the exponent (7.6) and its argument reduction (5), per species
    the Gibbs energy, shift and reduction (19) and the Newton mixture
    polynomial (14), per cell 200.  ncu: 2004 per evaluation against 1951."""
    return 12.6 * nr + 33.0 * ns + 200.0


def fine_flops_per_substep(ns: int, nr: int, M1: int, Y: int, rates32: bool = False,
                           alu: int = 1) -> float:
    """FP64 flops of one fine substep of the multirate chain per cell: one
    reaction-term evaluation (Newton solve included) and the update of
    eq. mrupdate, NV (2 + 2 (M1 + 1)) + ns (2 + 2 Y)."""
    nv = 5 + ns
    chem = chem_flops_per_eval_rates32(ns, nr) if rates32 else chem_flops_per_eval(ns, nr, alu)
    return chem + nv * (2 + 2 * (M1 + 1)) + ns * (2 + 2 * Y)


PRECISION_TEXT = {
    "fp64": "fp64",
    "mixed": ("mixed: FP32 stencil, flux and transport arithmetic; FP64 temperature, Gibbs "
              "energies, exponentials, rates and SDC accumulation"),
    "mixed_rates32": ("mixed with FP32-mantissa rates: as mixed, but the exponentials after their "
                      "FP64 argument reduction, the concentration products and the rate sums in FP32"),
}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def pipe_peaks(local: int) -> dict:
    """FMA-pipe throughputs of this GPU, measured now by smc_fma_throughput
    (FP64, FP32, paired FP32), with the SM clock sampled while they run.
    Iteration counts give about 0.3 s per pipe at the expected rates."""
    from paper_1309_7327_gb300 import smc
    sampler = ClockSampler(local)
    sampler.start()
    out = {}
    for name, kind, iters in (("fp64", 0, 150_000), ("fp32", 1, 8_000_000),
                              ("fp32x2", 2, 4_000_000), ("fp64_one_lane", 3, 150_000)):
        smc.smc_fma_throughput(kind, max(1, iters // 10))
        fl, ms, sms = smc.smc_fma_throughput(kind, iters)
        out[name + "_tflops"] = fl / 1e12
        out[name + "_ms"] = ms
        out["sm_count"] = sms
    out["clocks"] = sampler.stop()
    out["how"] = ("smc_fma_throughput: sm_count x 4 blocks x 256 threads, 8 independent FMA "
                  "chains per thread, CUDA events, after one untimed launch")
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures, keyed by (kernel, precision, workload): value, the capture it
# came from, and the SHA-256 (first 16 hex digits) of every source file the
# kernel is compiled from at the time of the capture.  A mismatch (the kernel
# changed since) makes the bench report traffic null.
_CHAIN_SRC = ["kernels_sdc.cu", "chem.cuh", "smc_internal.h"]
_MARCH_SRC = ["kernels_rhs.cu", "bc.cuh", "chem.cuh", "smc_internal.h"]
NCU_TRAFFIC = {
    # c4 at n = 64 (780 045 cells, state 162 MB > L2), the eight chain launches
    # of one step (four sweeps x two coarse intervals): mean 17 402 B per cell
    # and launch (profiles/k_fine_chain_fp64_c4_n64.md).  The same kernel
    # runs in both precisions (FP64 rates).
    ("k_fine_chain", "fp64", "c4"): {"bytes_per_cell": 17402.0, "files": _CHAIN_SRC,
                                     "digest": "5d726dc6735c98d5"},
    ("k_fine_chain", "mixed", "c4"): {"bytes_per_cell": 17402.0, "files": _CHAIN_SRC,
                                      "digest": "5d726dc6735c98d5"},
    # the per-face FP64 line kernel, x / y / z launches of one evaluation at
    # n = 64: 25.72 / 12.93 / 12.04 GB, mean 21 655 B per cell and launch
    # (profiles/k_march_fp64_c4_n64.md)
    ("k_march", "fp64", "c4"): {"bytes_per_cell": 21655.0, "files": _MARCH_SRC,
                                "digest": "a46a9b8d596b2980"},
}


def _sources_digest(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1309_7327_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, precision: str, workload: str, ncells_launch: float):
    """Measured DRAM bytes of one launch of `kernel` on this workload, or None
    when there is no capture or the kernel's sources changed since it."""
    e = NCU_TRAFFIC.get((kernel, precision, workload))
    if not e:
        return None
    try:
        if _sources_digest(e["files"]) != e["digest"]:
            return None
    except OSError:
        return None
    return e["bytes_per_cell"] * ncells_launch


def _oracle_worker(job):
    """One host process evaluating the oracle's right-hand side on a patch for
    `budget` seconds; returns (evaluations, seconds)."""
    patch, mech, dx, budget = job
    from oracle import rhs as orhs
    evals, t0 = 0, time.perf_counter()
    while True:
        orhs.rhs_ghosted(patch, mech, dx)
        evals += 1
        el = time.perf_counter() - t0
        if el > budget:
            return evals, el


def _host_cpu() -> str:
    """The host's architecture and CPU model (lscpu's, else /proc/cpuinfo's)."""
    import platform
    import subprocess
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{platform.machine()} {model}".strip()


def cpu_baseline(wl, budget_s: float = 15.0, all_cores_s: float = 0.0):
    """The oracle's right-hand side on a bounded sample of the workload's boxes
    (host cores, NumPy, single thread).  all_cores_s > 0: the same sample on
    every host core at once as well (one spawned process per core, each for
    that many seconds), reported beside the single-thread figure."""
    import numpy as np

    from oracle import rhs as orhs
    from oracle import thermo
    from paper_1309_7327_gb300 import synth
    g = wl.grid
    prim = synth.boxes_to_global(g, wl.prim)
    U = thermo.conserved(prim, wl.mech.nasa7, wl.mech.W)
    # one box's worth of cells (at most 32 per axis), evaluated as a ghosted
    # patch of the global field
    b = int(np.argmin([g.box_cells(i) for i in range(g.nboxes)]))
    (x0, y0, z0), (x1, y1, z1) = g.lo[b], g.hi[b]
    x1, y1, z1 = min(x1, x0 + 31), min(y1, y0 + 31), min(z1, z0 + 31)
    nz, ny, nx = U.shape[1:]
    iz = np.arange(z0 - 4, z1 + 5) % nz
    iy = np.arange(y0 - 4, y1 + 5) % ny
    ix = np.arange(x0 - 4, x1 + 5) % nx
    patch = U[:, iz][:, :, iy][:, :, :, ix]
    cells = (x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1)
    evals, t0 = 0, time.perf_counter()
    while True:
        orhs.rhs_ghosted(patch, wl.mech, g.dx)
        evals += 1
        el = time.perf_counter() - t0
        if el > budget_s or evals >= 50:
            break
    out = {"value": cells * evals / el / 1e6, "unit": "Mcell-RHS/s", "cores": 1,
           "kind": "oracle", "host": _host_cpu(),
           "sample": f"{evals} full RHS evaluations of {cells} cells of box {b} of workload "
                     f"{wl.name} by the NumPy FP64 oracle, {el:.1f} s"}
    if all_cores_s > 0:
        # spawned (not forked) processes: the parent may hold a CUDA context;
        # a worker that cannot start ends the pool with an error, not a hang
        import concurrent.futures as cf
        import multiprocessing as mp
        n = os.cpu_count() or 1
        try:
            with cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
                res = list(ex.map(_oracle_worker, [(patch, wl.mech, g.dx, all_cores_s)] * n,
                                  timeout=120 + 4 * all_cores_s))
            out["all_cores"] = {"value": sum(cells * e / t for e, t in res) / 1e6, "cores": n,
                                "sample": f"the same patch on {n} processes at once, "
                                          f"{all_cores_s:.0f} s each"}
        except Exception as e:                        # reported, never fatal
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out


def bench_config(wl, args, main_key, world):
    """The workload description both arms print."""
    nodes, sweeps, rsub = wl.nodes, wl.sweeps, wl.reaction_substeps
    M1 = nodes - 1
    per = rsub - 1 if rsub >= 2 else 0
    ncells, nv = wl.grid.ncells, 5 + wl.mech.ns
    if per and args.mr_mode == 2:
        M2 = M1 * per * max(args.fine_repeat, 1)
        return {"workload": args.workload + (f" (n={args.n})" if args.n else ""),
                "boxes": wl.grid.nboxes, "cells": ncells,
                "species": wl.mech.ns, "reactions": wl.mech.nr,
                "boundaries": "x outflow, y z periodic" if wl.x_outflow else "periodic",
                "integrator": (f"MRSDC mode 2: reactions implicit (BDF, rtol 1e-8) on {nodes} coarse "
                               f"GL nodes, advection-diffusion on {rsub} fine GL nodes per coarse "
                               f"interval, {sweeps} sweeps"),
                "rhs_evals_per_step": sweeps * M2,
                "reaction_evals_per_step": "adaptive (bdf_evals in the stats)",
                "precision": PRECISION_TEXT[main_key],
                "l2": "inputs larger than L2 (state %.0f MB)" % (nv * ncells * 8 / 1e6),
                "parallelism": "replicas" if world > 1 else "single GPU"}
    return {"workload": args.workload + (f" (n={args.n})" if args.n else ""),
            "boxes": wl.grid.nboxes, "cells": ncells,
            "species": wl.mech.ns, "reactions": wl.mech.nr,
            "boundaries": "x outflow, y z periodic" if wl.x_outflow else "periodic",
            "integrator": ((f"MRSDC {nodes} coarse / {rsub} fine GL"
                            + (f" x {args.fine_repeat} (type c)" if args.fine_repeat > 1 else " (type b)")
                            + f", {sweeps} sweeps") if rsub >= 2 else f"SDC {nodes} GL, {sweeps} sweeps")
                           + (f", residual exit eps = {args.sdc_exit}" if args.sdc_exit > 0 else ""),
            "rhs_evals_per_step": sweeps * M1,
            "reaction_evals_per_step": sweeps * M1 * per * max(args.fine_repeat, 1) if per else 0,
            "precision": PRECISION_TEXT[main_key],
            "l2": "inputs larger than L2 (state %.0f MB)" % (nv * ncells * 8 / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    """The oracle on the host cores (reference arm)."""
    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    from paper_1309_7327_gb300 import synth
    wl = synth.workload(args.workload, seed=args.seed, n=args.n)
    main_key = {"both": "fp64", "fp64+mixed": "fp64"}.get(args.precision, args.precision)
    for _ in range(args.warmup):
        cpu_baseline(wl, budget_s=1.0)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(wl, budget_s=5.0)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "Mcell-RHS/s (21 species)", "value": value,
            "unit": "Mcell-RHS/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic", "config": bench_config(wl, args, main_key, world),
            "cpu_baseline": dict(last, value=value),
            "e2e": {"value": value, "unit": "Mcell-RHS/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_heat(args):
    """The App. A heat problems (T1/T2) through smc_heat2d: narrow stencil and
    SDC (3 Gauss-Lobatto nodes, 4 sweeps) on an N x N periodic grid."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc, synth
    N = args.n or 4096
    f = synth.heat_fields(args.workload.upper(), N)
    dev = torch.device("cuda", 0)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)        # noqa: E731
    a, b, u = t(f["a"]), t(f["b"]), t(f["u0"])
    G = t(f["G"]) if f["G"] is not None else None
    h = f["h"]
    # the App. A stability rule, dt0 = 0.4 / ((dx^-2 + dy^-2) max(a, b))
    dt = 0.4 / ((2.0 / h ** 2) * max(float(f["a"].max()), float(f["b"].max())))
    smc.smc_heat2d(N, h, a, b, G, u, 0.0, dt, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.start()
    e0.record()
    nev = smc.smc_heat2d(N, h, a, b, G, u, 0.0, dt, args.steps)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    evals = nev - 1                            # the first call of each run evaluates F(U_0)
    value = N * N * evals / (ms / 1e3) / 1e6
    arrays = 5 if G is not None else 4         # a, b, u (, G) read and F written per evaluation
    per_step = 8 * arrays * 8 + 8 * 7 * 8      # evaluations + node updates (5 F sources, U in, U out)
    bytes_ = N * N * per_step * args.steps
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    # FP64 work of one evaluation per cell, each face counted once: a face is
    # 7 differences, 44 + 8 FMAs (the banded 8 x 8 narrow matrix), and a cell
    # takes two faces (x, y), two face differences, one sum (+ the source)
    face = 7 + 2 * (44 + 8)
    flops_eval = N * N * (2 * face + 3 + (2 if G is not None else 0))
    pk = pipe_peaks(0)
    fp64_peak = pk["fp64_tflops"] * 1e12
    fl_s = flops_eval * evals / (ms / 1e3)
    # ncu DRAM bytes of one k_heat_rhs launch (a 2048^2 capture scaled by cells)
    heat_traffic = ncu_traffic("k_heat_rhs", "fp64", args.workload, N * N)
    line = {"metric": f"Mcell-RHS/s (heat {args.workload.upper()})", "value": value,
            "unit": "Mcell-RHS/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": f"{N}x{N} periodic",
                       "integrator": "SDC 3 GL, 4 sweeps", "stencil": "8th-order narrow (SMC)",
                       "l2": "state and coefficients larger than L2 (%.0f MB)" % (N * N * 8 * 5 / 1e6)},
            "roofline": {"bound": "alu", "kernel": "whole step (k_heat_rhs + k_combo), FP64 flops of "
                                                    "the evaluations",
                         "achieved": fl_s / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                         "frac": fl_s / fp64_peak, "traffic": None,
                         "peak_source": "FP64 pipe, measured in this run by smc_fma_throughput "
                                        "(of measured)"},
            "hbm": {"kernel": "whole step", "algorithmic_bytes_per_step": N * N * per_step,
                    "achieved_gbs": bytes_ / (ms / 1e3) / 1e9, "peak_gbs": peak,
                    "frac": bytes_ / (ms / 1e3) / 1e9 / peak,
                    "k_heat_rhs_dram_bytes_per_launch": heat_traffic},
            "clocks": clocks, "pipe_peaks": pk, "gpu_launches": int(2 * evals)}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("t1", "t2"):
        run_heat(args)
        return
    if args.workload == "peaks":
        import torch

        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(0)
        pk = pipe_peaks(0)
        print(json.dumps({"metric": "FMA pipe throughput", "value": pk["fp64_tflops"],
                          "unit": "TFLOP/s (FP64)", "n_gpus": 1, "higher_is_better": True,
                          "data": "synthetic", "config": {"workload": "peaks"}, "pipe_peaks": pk,
                          "hbm_gbs": measured_peaks().get("hbm_gbs")}))
        return
    import numpy as np
    import torch

    import __graft_entry__
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc, synth

    wl = synth.workload(args.workload, seed=args.seed, n=args.n)
    nodes, sweeps, rsub = wl.nodes, wl.sweeps, wl.reaction_substeps
    M1 = nodes - 1
    evals_per_step = sweeps * M1
    if args.mr_mode == 2 and rsub >= 2:
        evals_per_step = sweeps * M1 * (rsub - 1) * max(args.fine_repeat, 1)
    ncells = wl.grid.ncells
    nv = 5 + wl.mech.ns

    variants = {"fp64": {"precision": 0}, "mixed": {"precision": 1},
                "mixed_rates32": {"precision": 1, "rates": 1}}
    for v in variants.values():
        if args.fine_repeat > 1:
            v["fine_repeat"] = args.fine_repeat
        if args.sdc_exit > 0:
            v["sdc_exit"] = args.sdc_exit
        if args.mr_mode == 2:
            v["mr_mode"] = 2

    def measure(name: str):
        """Warm up, then time args.steps steps on device-resident state."""
        opts = variants[name]
        precision = opts["precision"]
        torch.cuda.empty_cache()              # earlier variants' tensors
        h = smc.Smc(wl.grid, wl.mech, opts, x_outflow=wl.x_outflow)
        stream = torch.cuda.Stream(device)
        h.set_stream(stream)
        prim = torch.from_numpy(wl.prim).to(device)
        U = torch.empty_like(prim)
        with torch.cuda.stream(stream):
            h.prim_to_cons(prim, U)
        h.synchronize()
        del prim
        torch.cuda.empty_cache()              # the library allocates with cudaMalloc
        U0 = U.cpu()                          # the initial state, kept on the host
        def rhs_ms(reps=3):
            """CUDA-event time of one full right-hand-side evaluation."""
            F = torch.empty_like(U)
            h.rhs(U, F)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(device)
            a.record(stream)
            for _ in range(reps):
                h.rhs(U, F)
            b.record(stream)
            torch.cuda.synchronize(device)
            del F
            torch.cuda.empty_cache()
            return a.elapsed_time(b) / reps

        rhs_default = rhs_ms()                # the library's default schedule
        if args.tiles:                        # a fixed schedule (profiling runs)
            seg, xl, mv, *pers = (int(v) for v in args.tiles.split(","))
            pers = pers[0] if pers else 0
            h.set_option("segment", seg)
            h.set_option("x_layout", xl)
            h.set_option("march", mv)
            h.set_option("persistent", pers)
            tuned = {"segment": seg, "x_layout": xl, "march": mv, "persistent": pers}
        else:
            tuned = h.autotune(U)             # segment length, x-line layout, line kernel
        tuned = dict(tuned, rhs_ms_default=rhs_default, rhs_ms_tuned=rhs_ms())
        for _ in range(args.warmup):          # also fills the recycled f(U_0)
            h.sdc_step(U, wl.dt, nodes, sweeps, rsub)
        h.synchronize()
        base = h.stats()
        sampler = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(device)
        sampler.start()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):           # recycled steps: CUDA-graph replays
            h.sdc_step(U, wl.dt, nodes, sweeps, rsub)
        t_end.record(stream)
        torch.cuda.synchronize(device)
        clocks = sampler.stop()
        barrier(world)
        h.synchronize()
        ms = max_over_ranks(world, t_start.elapsed_time(t_end), device)
        st = h.stats()
        launches = {k: st["launches"][k] - base["launches"][k] for k in st["launches"]}
        evals_done = (st["n_rhs"] - base["n_rhs"]) / args.steps      # RHS evaluations per step
        bdf_evals = st["bdf_evals"] - base["bdf_evals"]
        # the same steps again with every launch timed by CUDA events (eager
        # launches): per-kernel durations for the rooflines
        h.set_option("profile", 1)
        for _ in range(args.steps):
            h.sdc_step(U, wl.dt, nodes, sweeps, rsub)
        h.synchronize()
        st2 = h.stats()
        h.set_option("profile", 0)
        # the same steps launched kernel by kernel (no graph replay), timed
        # like the graph-replayed ones: what the graph capture saves
        ms_eager = None
        if not args.lean:
            h.set_option("use_graphs", 0)
            h.sdc_step(U, wl.dt, nodes, sweeps, rsub)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(device)
            e0.record(stream)
            for _ in range(args.steps):
                h.sdc_step(U, wl.dt, nodes, sweeps, rsub)
            e1.record(stream)
            torch.cuda.synchronize(device)
            ms_eager = e0.elapsed_time(e1) / args.steps
        h.close()
        return dict(ms_step=ms / args.steps, launches=launches, kms=st2["kernel_ms"],
                    clocks=clocks, U0=U0, tuned=tuned, ms_eager=ms_eager, evals=evals_done,
                    bdf_evals=bdf_evals)

    def end_to_end(name, tuned, U0):
        """The variant end to end through the C ABI: a pinned host buffer, with
        the host->device and device->host copies of every step inside the timed
        region.  Seconds per step and the clocks seen meanwhile."""
        Uh = U0.cpu().clone().pin_memory()
        torch.cuda.empty_cache()              # the measured run's tensors
        h2 = smc.Smc(wl.grid, wl.mech, dict(variants[name], segment=tuned["segment"],
                                            x_layout=tuned["x_layout"], march=tuned["march"],
                                            persistent=tuned["persistent"]),
                     x_outflow=wl.x_outflow)
        h2.sdc_step(Uh, wl.dt, nodes, sweeps, rsub)
        e2e_steps = max(1, min(args.steps, 3))
        barrier(world)
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            h2.sdc_step(Uh, wl.dt, nodes, sweeps, rsub)
        sec = (time.perf_counter() - t0) / e2e_steps
        clocks = sampler.stop()
        h2.close()
        return max_over_ranks(world, sec, device), clocks

    pk = pipe_peaks(local)                    # FMA-pipe denominators, measured now
    runs = {}
    order = {"both": ["fp64", "mixed", "mixed_rates32"],
             "fp64+mixed": ["fp64", "mixed"]}.get(args.precision, [args.precision])
    for name in order:
        runs[name] = measure(name)
        if name == order[0]:
            # the headline variant end to end, in the same GPU state as its
            # device-resident measurement
            e2e_s, e2e_clocks = end_to_end(name, runs[name]["tuned"], runs[name]["U0"])
    main_key = order[0]
    R = runs[main_key]
    ms_step, launches, kms, clocks, U0 = R["ms_step"], R["launches"], R["kms"], R["clocks"], R["U0"]
    if args.sdc_exit > 0:                     # sweeps end early: count what ran
        evals_per_step = R["evals"]
    value = job_throughput(world, ncells, evals_per_step, ms_step)
    main_opts = variants[main_key]

    # rooflines of the two heaviest kernels; "roofline" is the one with the
    # larger share of the step
    fp64_peak = pk["fp64_tflops"] * 1e12
    # the mixed line kernels issue paired FP32 FMAs: their pipe peak is the
    # larger of the plain and paired measurements
    fp32_peak = max(pk["fp32_tflops"], pk["fp32x2_tflops"]) * 1e12
    src64 = "FP64 pipe, measured in this run by smc_fma_throughput (of measured)"
    src32 = "FP32 pipe (paired FMAs), measured in this run by smc_fma_throughput (of measured)"
    rooflines = {}
    n_march = launches["march"]
    if wl.x_outflow:
        # the kernel class also holds one launch per evaluation for the cells
        # next to the x ends (lowered stencils): count the three direction
        # launches only, their time keeping that small launch's share
        n_march = n_march * 3 // 4
    if n_march:
        march_ms = kms["march"] / n_march
        if main_opts["precision"] == 0:
            fl, peak, src = march_flops_per_cell(wl.mech.ns) * ncells, fp64_peak, src64
        else:
            fl, peak, src = march_flops_per_cell_mixed(wl.mech.ns) * ncells, fp32_peak, src32
        rooflines["k_march"] = {
            "bound": "alu", "kernel": "k_march (one stencil direction)",
            "achieved": fl / (march_ms / 1e3) / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": fl / (march_ms / 1e3) / peak,
            "traffic": ncu_traffic("k_march", main_key, args.workload, ncells),
            "peak_source": src,
            "share": kms["march"] / max(sum(kms.values()), 1e-9)}
        # the same kernel against HBM: algorithmic bytes = every primitive
        # plane read once over the ghosted cells plus the accumulator written
        # once over the interior cells
        esize, planes = (8, 17 + 6 * wl.mech.ns) if main_opts["precision"] == 0 else \
            (4, 28 + 9 * wl.mech.ns)
        ghosted = sum((wl.grid.box_shape(b)[0] + 8) * (wl.grid.box_shape(b)[1] + 8)
                      * (wl.grid.box_shape(b)[2] + 8) for b in range(wl.grid.nboxes))
        mbytes = planes * esize * ghosted + nv * esize * ncells
        hbm_peak_m = measured_peaks().get("hbm_gbs", 6800.0)
        rooflines["k_march"]["hbm"] = {
            "algorithmic_bytes": mbytes, "achieved_gbs": mbytes / (march_ms / 1e3) / 1e9,
            "peak_gbs": hbm_peak_m, "frac": mbytes / (march_ms / 1e3) / 1e9 / hbm_peak_m}
    alu = int(main_opts.get("alu", 1))        # SMC_OPT_ALU (library default 1)
    n_fine = launches["fine"]
    if n_fine:
        per = rsub - 1
        fine_ms = kms["fine"] / n_fine
        rates32 = main_opts.get("rates", 0) == 1
        fl = fine_flops_per_substep(wl.mech.ns, wl.mech.nr, M1, rsub, rates32=rates32,
                                    alu=alu) * ncells * per
        rooflines["k_fine_chain"] = {
            "bound": "alu", "kernel": "k_fine_chain (reaction substeps of one coarse interval)",
            "achieved": fl / (fine_ms / 1e3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": fl / (fine_ms / 1e3) / fp64_peak,
            "traffic": ncu_traffic("k_fine_chain", main_key, args.workload, ncells),
            "peak_source": src64,
            "share": kms["fine"] / max(sum(kms.values()), 1e-9)}
        if alu and not rates32:
            # the same work counted as the FP64 operations of the FP64-pipe
            # exponentials it replaces
            fl_eq = fine_flops_per_substep(wl.mech.ns, wl.mech.nr, M1, rsub, alu=0) * ncells * per
            rooflines["k_fine_chain"]["fp64_equivalent"] = {
                "achieved": fl_eq / (fine_ms / 1e3) / 1e12,
                "frac": fl_eq / (fine_ms / 1e3) / fp64_peak,
                "note": "achieved/frac count the FP64-pipe flops; here the exponentials, which "
                        "run on the integer and FP32 pipes, are counted as the 14 FP64 flops each "
                        "they replace"}
    if launches.get("bdf"):
        bdf_ms = kms["bdf"] / launches["bdf"]
        evals_launch = R["bdf_evals"] / launches["bdf"]
        fl = chem_flops_per_eval(wl.mech.ns, wl.mech.nr, alu) * evals_launch
        rooflines["k_react_bdf"] = {
            "bound": "alu", "kernel": "k_react_bdf (implicit reactions over one coarse interval)",
            "achieved": fl / (bdf_ms / 1e3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": fl / (bdf_ms / 1e3) / fp64_peak, "traffic": None,
            "note": "production-rate flops of the counted evaluations only (Jacobian, LU and "
                    "temperature solves not counted): a lower bound",
            "peak_source": src64,
            "share": kms["bdf"] / max(sum(kms.values()), 1e-9)}
    roofline = max(rooflines.values(), key=lambda r: r["share"]) if rooflines else None
    # HBM-bound stage: SDC / fine-node updates
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    per = rsub - 1 if rsub >= 2 else 0
    M1 = nodes - 1
    if per and launches["fine"]:
        bytes_fine = ncells * 8 * (2 * nv + per * (M1 + 3) * nv + per * (rsub + 2) * wl.mech.ns)
        fine_ms = kms["fine"] / max(launches["fine"], 1)
        hbm = {"kernel": "k_fine_chain", "achieved_gbs": bytes_fine / (fine_ms / 1e3) / 1e9,
               "peak_gbs": hbm_peak, "frac": bytes_fine / (fine_ms / 1e3) / 1e9 / hbm_peak,
               "note": "algorithmic bytes; the chain also evaluates reactions in FP64"}
    else:
        hbm = None
    # the fused right-hand side alone (every stage of one evaluation: gather,
    # primitives, transport, stencils, correction terms, reactions) against
    # HBM: its algorithmic bytes are U read once and dUdt written once
    rhs_ms = R["tuned"]["rhs_ms_tuned"]
    rhs_bytes = 2 * nv * 8 * ncells
    rhs_stage = {"ms_per_evaluation": rhs_ms, "algorithmic_bytes": rhs_bytes,
                 "achieved_gbs": rhs_bytes / (rhs_ms / 1e3) / 1e9,
                 "peak_gbs": hbm_peak, "frac_hbm": rhs_bytes / (rhs_ms / 1e3) / 1e9 / hbm_peak,
                 "note": "one full RHS evaluation (CUDA events, autotuned schedule); the stage is "
                         "bound by the FP64 (or FP32) pipe, not by HBM: see rooflines"}
    mode2_note = None
    if args.mr_mode == 2:
        mode2_note = ("MRSDC mode 2 sweeps converge while |r| dt_p <= ~250 (r the reaction "
                      "eigenvalue, dt_p the coarse interval); with the paper's Lobatto nodes the "
                      "converged sweeps are accurate only while |r| dt_p is a few (A- but not "
                      "L-stable collocation)")
    precision_report = {k: {"value": world * ncells * evals_per_step / (r["ms_step"] / 1e3) / 1e6,
                            "ms_per_step": r["ms_step"], "autotuned": r["tuned"],
                            "ms_per_step_without_graphs": r["ms_eager"],
                            "kernel_ms_per_step": {kk: vv / args.steps for kk, vv in r["kms"].items()}}
                        for k, r in runs.items()}
    if "mixed" in runs and "fp64" in runs:
        precision_report["mixed_speedup_vs_fp64"] = runs["fp64"]["ms_step"] / runs["mixed"]["ms_step"]
        # the error that speedup comes at: one right-hand side of the initial
        # state in each precision, per component max|F_mixed - F_fp64| / max|F_fp64|
        torch.cuda.empty_cache()
        Ud = U0.to(device)
        F = {}
        for key, prec in (("fp64", 0), ("mixed", 1)):
            with smc.Smc(wl.grid, wl.mech, {"precision": prec}, x_outflow=wl.x_outflow) as he:
                F[key] = torch.empty_like(Ud)
                he.rhs(Ud, F[key])
                he.synchronize()
        num = (F["mixed"] - F["fp64"]).abs().amax(dim=1)
        den = F["fp64"].abs().amax(dim=1).clamp_min(1e-300)
        precision_report["mixed_rhs_error_vs_fp64"] = float((num / den).max())
        del Ud, F
    if "mixed_rates32" in runs and "fp64" in runs:
        precision_report["mixed_rates32_speedup_vs_fp64"] = (runs["fp64"]["ms_step"]
                                                             / runs["mixed_rates32"]["ms_step"])

    # end to end (measured right after the headline variant, above)
    e2e = {"value": world * ncells * evals_per_step / e2e_s / 1e6, "unit": "Mcell-RHS/s",
           "h2d_bytes_per_step": nv * ncells * 8, "d2h_bytes_per_step": nv * ncells * 8,
           "host_buffer": "pinned", "clocks": e2e_clocks}

    if rank == 0:
        cpu = cpu_baseline(wl, all_cores_s=8.0) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": "Mcell-RHS/s (21 species)", "value": value, "unit": "Mcell-RHS/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if main_key == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": bench_config(wl, args, main_key, world),
            "roofline": roofline, "rooflines": rooflines, "hbm": hbm, "rhs_stage": rhs_stage,
            "pipe_peaks": pk, "cpu_baseline": cpu, "e2e": e2e,
            "precisions": precision_report,
            "gpu_launches": int(sum(launches.values())),
            "kernel_ms_per_step": {k: kms[k] / args.steps for k in kms},
            "clocks": clocks,
        }
        if mode2_note:
            line["mode2_stiffness_bound"] = mode2_note
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
