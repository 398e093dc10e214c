#!/usr/bin/env python3
"""Benchmark of the multigrid pressure-Poisson path inside the projection
step (Algorithm 1), GB300.

Headline workload (default ``--config ns2d``): incompressible flow past a
square block, 2048 x 1024 cells (h = 1), a 64 x 64 solid block centred at
(512, 512), inflow u = 1, nu = 0.64 (Re = 100 on the block side),
dt = 0.1, initial velocity = inflow + 1% seeded Gaussian noise (seed 0).  One
bench step = one full projection step: two-pass momentum, divergence RHS,
the pressure-correction solve to relative residual 1e-6 (float64 iterate)
and the velocity/pressure correction.  Metric: solved pressure unknowns
(fluid cells) per second.

Other configs (``--config``): ``poisson2d`` (256^2, 8 blobs, zero
Dirichlet), ``poisson3d`` (256^3, 8 blobs; ``--prec fp32|fp16|bf16``),
``ns3d`` (256 x 128 x 128, 32^3 cube), ``batched`` (1024 uneven 2D
instances) and ``timing3d`` (the paper's timing workload of Sec. 3.4: flow
past a cube in an n^3 domain, ``--size 128|256|512``, 20 multigrid
iterations per time step with the finite-element filters; metric: seconds
for five time steps); ``advdiff`` (one implicit advection-diffusion step
of Sec. 3.2: 128^2 nodes, upwind, C = 50, ``--ad-size 128|1024|4096``;
V(2,2) cycles to relres 1e-6, or ``--cycle sawtooth`` for the paper's form
stopped on the L1 change 1e-5).

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (each step one oracle step of a bounded
sample of the workload).
"""
import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2402_17913_gb300 import inputs as I  # noqa: E402

METRIC = "solved unknowns/sec to 1e-6 rel residual"
TIMING_METRIC = "seconds for 5 time steps of the 3D flow past a cube"
AD_L1_METRIC = "solved unknowns/sec to an L1 change of 1e-5 per cycle"
UNIT = "unknowns/s"
TOL = 1e-6

# Batched solve: bytes per fine cell of one CG iteration (the four fine
# passes below, plus one cell byte in three of them, plus about a third more
# for the coarser levels) and of one float-float refinement pass.
BATCH_ITER_BYTES = 72
OUTER_BYTES = 28
KERNEL_CLASSES = ("down_fine", "up_fine", "p_update", "xr_update", "outer")


def algo_bytes_per_cell(cls, dim, prec="fp32", masked=False):
    """Algorithmic bytes per fine-grid cell of one launch of kernel class
    `cls` (the method's own minimum: each array read or written once per
    launch, at its own storage width).  The level arrays (the finest
    iterate x and every coarser level's arrays) are 4 bytes in float32 and 2
    in FP16/BF16; the finest right-hand side (the CG residual r) and output
    z, and the CG vectors, are float32 in every form; a masked grid reads one
    cell byte per cell in the level kernels; the coarse level has 1/2^dim of
    the cells."""
    t = 4 if prec == "fp32" else 2
    c = 1.0 / (1 << dim)
    m = 1 if masked else 0
    return {
        "down_fine": 4 + t + t * c + m,      # read b; write x, coarse b
        "up_fine": 4 + t + t * c + 4 + m,    # read b, x, coarse e; write z
        "p_update": 4 + 4 + 4,               # read z, p_old; write p ((p, A p) reduced)
        "xr_update": 4 + 8 + 8,              # read p; read+write d, r (A p formed from p)
        "outer": 4 + 8 + 4 + 8 + 4,          # read b, iterate, d; write iterate, r
    }[cls]


# Bytes per cell a solve keeps live (the right-hand side and its copy, the
# iterate, the CG vectors, the refinement pair, about a third more for the
# coarser levels): a grid below L2 / this stays L2-resident between launches.
LIVE_BYTES_PER_CELL = 48


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="poisson3d",
                    choices=["ns2d", "ns3d", "poisson2d", "poisson3d", "batched", "timing3d", "advdiff"])
    ap.add_argument("--ad-size", type=int, default=128, choices=[128, 1024, 4096],
                    help="advdiff: nodes per side")
    ap.add_argument("--size", type=int, default=256, choices=[128, 256, 512],
                    help="timing3d: cells per side of the cubic domain")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--guess", default="zero", choices=["zero", "net"],
                    help="ns3d: initial guess of each pressure solve (net = the learned guess, trained in the run)")
    ap.add_argument("--cycle", default="v", choices=["v", "sawtooth"],
                    help="poisson2d/3d: V(2,2)-preconditioned CG (default) or the paper's sawtooth cycle")
    ap.add_argument("--stencil", default="fd", choices=["fd", "fe"],
                    help="ns2d/ns3d: momentum filters, 5/7-point (default) or the finite-element 9/27-point ones")
    ap.add_argument("--guess-level", type=int, default=1, choices=[0, 1, 2],
                    help="ns3d --guess net: the network runs on the grid coarsened this many times")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch-count", type=int, default=1024,
                    help="batched: instances in the batch (the workload has 1024; fewer for profiling captures)")
    ap.add_argument("--advance", type=int, default=None,
                    help="ns2d/ns3d: untimed steps from the seeded initial state before the warm-up "
                         "(default: ns2d 480, ns3d 180, so that the timed steps end near step 500 / 200)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-timed", action="store_true",
                    help="run warm-up and timed steps only (for launch-list captures)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workloads
FILTERS = {False: "5/7-point (App. A)", True: "finite-element 9/27-point (App. A)"}


class NS2D:
    name = "ns2d_block_2048x1024"
    dim = 2

    def __init__(self, scale=1, fe=False):
        self.fe = fe
        self.cells = (2048 // scale, 1024 // scale)
        self.block = 64 // scale
        self.centre = (512 // scale, 512 // scale)
        self.nu, self.dt, self.uin = 0.64 / scale, 0.1, 1.0
        self.solid = I.block_mask(self.cells, self.centre, self.block)
        self.units = int((~self.solid).sum())

    def config(self):
        return {"workload": "2D projection step, flow past a square block", "cells": list(self.cells),
                "block": self.block, "nu": self.nu, "dt": self.dt, "u_inflow": self.uin,
                "solve_rel_tol": TOL, "unknowns_per_step": self.units,
                "momentum_filters": FILTERS[self.fe], "l2": "256 MiB buffer written between timed steps",
                "timed_steps": list(getattr(self, "window", ()))}


class NS3D:
    """3D flow past a cube: 256 x 128 x 128 cells (h = 1), a 32^3 solid cube
    centred at (64, 64, 64), inflow u = 1, nu = 0.32 (Re = 100 on the cube
    side), dt = 0.1, initial velocity = inflow + 1% noise (seed 0)."""
    name = "ns3d_cube_256x128x128"
    dim = 3

    def __init__(self, scale=1, fe=False):
        self.fe = fe
        self.cells = (256 // scale, 128 // scale, 128 // scale)
        self.block = 32 // scale
        self.centre = (64 // scale, 64 // scale, 64 // scale)
        self.nu, self.dt, self.uin = 0.32 / scale, 0.1, 1.0
        self.solid = I.block_mask(self.cells, self.centre, self.block)
        self.units = int((~self.solid).sum())

    def config(self):
        return {"workload": "3D projection step, flow past a cube", "cells": list(self.cells), "block": self.block,
                "nu": self.nu, "dt": self.dt, "u_inflow": self.uin, "solve_rel_tol": TOL,
                "unknowns_per_step": self.units, "momentum_filters": FILTERS[self.fe],
                "l2": "256 MiB buffer written between timed steps", "timed_steps": list(getattr(self, "window", ()))}


class Timing3D:
    """The timing workload of Sec. 3.4 (the paper's timing table): flow past
    a cube in an n^3 domain (h = 1), the cube 10/128 of the side, centred at
    (n/4, n/2, n/2) as in the paper's 128^3 case, Re = 200 on the cube side
    (nu = side / 200), dt = 0.1, the fluid at rest with u = 1 on the inflow
    faces and the finite-element 27-point filters.  Pressure solve: the
    paper's form, a fixed 20 stationary sawtooth cycles per time step with no
    tolerance (``--cycle sawtooth``), or this library's default solve,
    V(2,2)-preconditioned CG with float-float refinement to relres 1e-6
    (``--cycle v``; its iteration count is reported)."""
    dim = 3
    iters = 20
    # the paper's seconds for five steps x 20 iterations (Tesla T4; one
    # Xeon 2.3 GHz CPU), context only
    paper_s = {128: (3.0, 165.0), 256: (11.0, 1275.0), 512: (34.0, 14376.0)}

    def __init__(self, n=256, cycle="sawtooth", scale=1):
        self.fe = True
        self.cycle = cycle
        n = n // scale
        self.n = n
        self.name = "ns3d_timing_%d" % n
        self.cells = (n, n, n)
        self.block = max(2, round(10 * n / 128))
        self.centre = (n // 4, n // 2, n // 2)
        self.nu, self.dt, self.uin = self.block / 200.0, 0.1, 1.0
        self.solid = I.block_mask(self.cells, self.centre, self.block)
        self.units = int((~self.solid).sum())

    def initial_velocity(self):
        q = [np.zeros((self.n, self.n, self.n + 1), np.float32), np.zeros((self.n, self.n + 1, self.n), np.float32),
             np.zeros((self.n + 1, self.n, self.n), np.float32)]
        q[0][..., 0] = self.uin
        return q

    def config(self):
        t4, cpu = self.paper_s.get(self.n, (None, None))
        return {"workload": "3D flow past a cube, five time steps x 20 multigrid iterations (the paper's timing table)",
                "cells": list(self.cells), "block": self.block, "centre": list(self.centre), "nu": self.nu,
                "dt": self.dt, "u_inflow": self.uin, "momentum_filters": FILTERS[True],
                "solver": ("20 stationary sawtooth cycles (coarse scale 1/2) per step" if self.cycle == "sawtooth"
                           else "V(2,2)-preconditioned CG to relres 1e-6 per step"),
                "paper_seconds_t4": t4, "paper_seconds_xeon_cpu": cpu,
                "l2": "256 MiB buffer written between timed steps"}


class AdvDiff:
    """One backward-Euler advection-diffusion step (Sec. 3.2): n^2 nodes
    (h = 1), (u, v) = (1, 1), nu = 2, dt = 50 (C = 50), upwind advection, a
    Gaussian of width 10 n / 128 at the centre as T^n and initial guess.
    ``cycle='v'``: V(2,2) cycles (omega 2/3, re-discretised coarse levels)
    to relres 1e-6; ``'sawtooth'``: the paper's form (Jacobi alpha = 1, one
    sweep, halved coarse correction) until the L1 change of one cycle is
    <= 1e-5."""
    dim = 2
    h, dt, nu, u, v = 1.0, 50.0, 2.0, 1.0, 1.0

    def __init__(self, n=128, cycle="v"):
        self.n, self.cycle = n, cycle
        self.name = "advdiff_%d" % n
        self.shape = (n, n)
        self.units = n * n
        self.gamma = 10.0 * n / 128.0

    def rhs(self):
        return I.advdiff_gaussian(self.shape, gamma=self.gamma).astype(np.float32)

    def config(self):
        return {"workload": "one implicit advection-diffusion step (upwind, C = 50) solved by multigrid",
                "nodes": [self.n, self.n], "u": self.u, "v": self.v, "nu": self.nu, "dt": self.dt,
                "gaussian_width": self.gamma,
                "solver": ("V(2,2) cycles to relres 1e-6" if self.cycle == "v"
                           else "sawtooth (alpha 1, one sweep, coarse scale 1/2) to L1 change 1e-5"),
                "l2": "256 MiB buffer written between timed steps"}


class Poisson:
    def __init__(self, shape, prec, cycle="v"):
        self.shape = shape
        self.dim = len(shape)
        self.prec = prec
        self.cycle = cycle
        self.units = int(np.prod(shape))
        self.name = "poisson%dd_%s_%s" % (self.dim, "x".join(map(str, shape)), prec)
        if cycle != "v":
            self.name += "_" + cycle

    def config(self):
        c = {"workload": "%dD pressure Poisson, 8 Gaussian blobs, zero Dirichlet" % self.dim,
             "shape": list(reversed(self.shape)), "solve_rel_tol": TOL, "inner_precision": self.prec,
             "unknowns_per_step": self.units, "l2": "256 MiB buffer written between timed steps"}
        if self.cycle == "sawtooth":
            c["cycle"] = "sawtooth (paper App. B), stationary, coarse scale 1/2, 2 post sweeps"
        return c


def shard_by_work(weights, world):
    """Split items over `world` ranks by work: heaviest first, each onto the
    rank with the least work so far (ties: the lowest rank).  Returns one
    sorted list of item indices per rank."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in sorted(range(len(weights)), key=lambda i: (-weights[i], i)):
        r = min(range(world), key=lambda j: (load[j], j))
        load[r] += weights[k]
        parts[r].append(k)
    return [sorted(p) for p in parts]


class Batched:
    """1024 independent square instances, sides uniform in {64, 128, 256,
    512} (seed 1234), random rectangle solids covering U(0, 0.1) of the
    cells (flood-filled), 8-blob right-hand sides (seed = instance index),
    zero Dirichlet faces.  Under several ranks the one batch is split by
    work (sum of N^2, heaviest instance first onto the least-loaded rank):
    each rank solves its share with no collective, and the whole job is the
    1024 instances (strong scaling)."""
    name = "batched_1024"  # the workload; config() states the instance count of a run
    dim = 2

    def __init__(self, count=1024, seed=1234, limit=None, rank=0, world=1):
        self.rank, self.world = rank, world
        sides, fracs, rng = I.batched_sides(count, seed)
        n_all = len(sides) if limit is None else min(limit, len(sides))
        self.count = n_all
        self.own = set(shard_by_work([sides[k] ** 2 for k in range(n_all)], world)[rank])
        self.index, self.shapes, self.spacings, self.solids, self.rhs = [], [], [], [], []
        self.job_units = 0
        for k in range(n_all):
            n, f = sides[k], fracs[k]
            solid = I.random_solid_mask((n, n), rng, f)  # every mask, in draw order
            self.job_units += int((~solid).sum())
            if k not in self.own:
                continue
            self.index.append(k)
            self.shapes.append((n, n))
            self.spacings.append((1.0 / (n + 1), 1.0 / (n + 1)))
            self.solids.append(solid)
            self.rhs.append(I.blob_rhs((n, n), k, solid=solid).astype(np.float32))
        self.units = int(sum((~s).sum() for s in self.solids))
        self.cells = int(sum(n * n for n, _ in self.shapes))

    def config(self):
        c = {"workload": "batched 2D Poisson, %d instances of sides {64,128,256,512}, random solids"
             % self.count, "cells": self.cells,
             "solve_rel_tol": TOL, "unknowns_per_step": self.units,
             "l2": "inputs (%.1f GB) larger than L2" % (self.cells * 60 / 1e9)}
        if self.world > 1:
            c["sharding"] = ("one batch split over %d ranks by sum of N^2 (heaviest first), no collective; "
                             "this rank: %d instances" % (self.world, len(self.shapes)))
        return c


PREC = {"fp32": 0, "fp16": 1, "bf16": 2}


# ---------------------------------------------------------------------------
class NvmlClocks:
    """Samples the SM clock, its maximum and the clock-event reasons of
    every GPU every 10 ms through NVML (read-only queries), in a thread."""
    # clock-event reason bits (nvml.h)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self):
        import ctypes
        import threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        n = ctypes.c_uint(0)
        lib.nvmlDeviceGetCount_v2(ctypes.byref(n))
        self.h = []
        for i in range(n.value):
            hd = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(i, ctypes.byref(hd)) == 0:
                self.h.append(hd)
        if not self.h:
            raise RuntimeError("no NVML device")
        self.lib, self.ct = lib, ctypes
        self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.sm, self.mx, self.reasons = [], [], set()
        self.stop = threading.Event()
        self.t = threading.Thread(target=self.run, daemon=True)
        self.t.start()

    def run(self):
        ct, lib = self.ct, self.lib
        while not self.stop.is_set():
            for hd in self.h:
                c, m, r = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
                if lib.nvmlDeviceGetClockInfo(hd, 1, ct.byref(c)) == 0:
                    self.sm.append(float(c.value))
                if lib.nvmlDeviceGetMaxClockInfo(hd, 1, ct.byref(m)) == 0:
                    self.mx.append(float(m.value))
                if self.reason_fn(hd, ct.byref(r)) == 0:
                    for name, bit in self.BITS.items():
                        if r.value & bit:
                            self.reasons.add(name)
            self.stop.wait(0.01)

    def summary(self):
        self.stop.set()
        self.t.join()
        self.lib.nvmlShutdown()
        return {"sm_mhz": statistics.median(self.sm) if self.sm else None,
                "sm_max_mhz": max(self.mx) if self.mx else None, "reasons": sorted(self.reasons),
                "samples": len(self.sm), "source": "NVML, 10 ms"}


def clocks_sampler():
    try:
        return NvmlClocks(), None, None
    except Exception:
        pass
    path = tempfile.mktemp(suffix=".csv")
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f, path
    except Exception:
        return None, None, path


def clocks_summary(p, f, path):
    if isinstance(p, NvmlClocks):
        return p.summary()
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    p.wait()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [t.strip() for t in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def l2_read_peak(L, dev, l2_size):
    """L2 read bandwidth (GB/s) of a streaming kernel on this GPU: a buffer
    of a quarter of L2 read 64 times in one launch (best of 5 launches,
    CUDA events)."""
    import torch
    n = (l2_size // 4 // 4) // 4 * 4
    buf = torch.ones(n, dtype=torch.float32, device=dev)
    sink = torch.empty(4 * torch.cuda.get_device_properties(dev).multi_processor_count, dtype=torch.float32,
                       device=dev)
    reps, best = 64, float("inf")
    L.mg_probe_l2_read(buf, reps, sink)
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.mg_probe_l2_read(buf, reps, sink)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return n * 4.0 * reps / (best * 1e-3) / 1e9


# The translation unit of the dominant kernel of each workload with a
# committed traffic summary; its hash also covers the headers it includes.
TRAFFIC_TU = {"ns2d_block_2048x1024": "mg_stream2d.cu", "poisson3d_256x256x256_fp32": "mg_tma3d.cu",
              "ns3d_cube_256x128x128": "mg_tma3d.cu"}
KERNEL_HEADERS = ["mg_kernels.cuh", "launch.h", "npmg_internal.cuh", "tma.cuh", "tma_host.h", "refine.cuh"]


def _code_only(text):
    """C/C++ source with comments removed and whitespace collapsed, so that
    a comment edit does not count as a change of the kernel."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_hash(tu=None):
    """Hash of the code a kernel is compiled from: translation unit `tu`
    with the level-kernel headers and the public header (every csrc file
    when tu is None), comments ignored."""
    csrc = os.path.join(ROOT, "paper_2402_17913_gb300", "csrc")
    if tu is None:
        paths = sorted(glob.glob(os.path.join(csrc, "*")))
    else:
        paths = [os.path.join(csrc, f) for f in [tu] + KERNEL_HEADERS] + [os.path.join(ROOT, "include", "npmg.h")]
    h = hashlib.sha256()
    for p in paths:
        h.update(_code_only(open(p, encoding="utf-8", errors="replace").read()).encode())
    return h.hexdigest()[:12]


def recorded_traffic(workload, cls):
    """DRAM bytes per launch of kernel class `cls` from the committed ncu
    summary, if it was taken on the current sources of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic_%s.md" % workload)
    if not os.path.exists(path) or workload not in TRAFFIC_TU:
        return None
    src = source_hash(TRAFFIC_TU[workload])
    for line in open(path):
        m = re.match(r"\s*traffic_bytes_per_launch:\s*(\w+)\s+([0-9.eE+]+)\s+src=(\w+)", line)
        if m and m.group(1) == cls and m.group(3) == src:
            return float(m.group(2))
    return None


# ---------------------------------------------------------------------------
# learned initial guess (3D flow): solver pairs from the seeded run, training
GUESS_PAIRS, GUESS_CROP, GUESS_BATCH, GUESS_LR = 5000, 64, 8, 1e-3


def train_guess(L, ns, wl, u, v, w, p, solid_t, train_steps, level):
    """Runs the seeded flow from its initial state, cutting each step's
    (b, p^n, dp) into crops until GUESS_PAIRS are stored, then trains the
    network on them with the residual loss; returns a dict with the handle
    and the training record.  At level 1 the fields are first restricted once
    (the network then runs on the coarsened grid) and crops are 32^3 with
    spacing 2."""
    import torch
    crop = GUESS_CROP >> level
    g = L.gn_create(I.convnet_weights(0, last_scale=1e-3))
    L.gn_dataset_reserve(g, (crop,) * 3, GUESS_PAIRS, float(1 << level))
    cells = tuple(c >> level for c in wl.cells)
    if level:
        nc = cells[0] * cells[1] * cells[2]
        coarse = [torch.empty(nc, dtype=torch.float32, device=p.device) for _ in range(3)]
        solid_c = torch.empty(nc, dtype=torch.uint8, device=p.device)
    t0 = time.perf_counter()
    gen_steps = 0
    while L.gn_dataset_size(g) < GUESS_PAIRS:
        L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, TOL, stats=False)
        if level:
            L.ns_coarse_fields(ns, level, p, coarse[0], coarse[1], coarse[2], solid_c)
            L.gn_dataset_add(g, cells, coarse[0], coarse[1], coarse[2], solid_c)
        else:
            b_ptr, dp_ptr = L.ns_last_fields(ns)
            L.gn_dataset_add(g, cells, b_ptr, p, dp_ptr, solid_t)
        gen_steps += 1
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = L.gn_train(g, train_steps, GUESS_BATCH, 1, GUESS_LR, L.GN_LOSS_RESIDUAL)
    t2 = time.perf_counter()
    L.ns_set_guess_level(ns, g, level)
    tail = float(np.mean(losses[-50:]))
    return {"handle": g, "level": level, "net_cells": list(cells), "pairs": GUESS_PAIRS, "crop": crop,
            "generation_steps": gen_steps,
            "generation_s": round(t1 - t0, 2), "train_steps": train_steps, "batch": GUESS_BATCH, "lr": GUESS_LR,
            "train_s": round(t2 - t1, 2), "loss_first50": float(np.mean(losses[:50])), "loss_last50": tail,
            "train_relres_last50": float(np.sqrt(2.0 * tail))}


def guess_report(L, guess, step_stats, ns, wl, u, v, w, p, compare=5):
    """Guess quality over the timed steps, then the same states solved from
    the guess and from zero side by side (iterations and device ms)."""
    import torch
    rel = [s["guess_relres"] for s in step_stats]
    rej = sum(s["guess_rejected"] for s in step_stats)
    pairs = []
    for _ in range(compare):
        state = [t.clone() for t in (u, v, w, p)]
        L.ns_set_guess_level(ns, guess["handle"], guess["level"])
        _, sg = L.ns_step(ns, state[0], state[1], state[2], state[3], wl.dt, wl.nu, wl.uin, TOL)
        L.ns_set_guess(ns, None)
        _, sz = L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, TOL)
        pairs.append((sg["iters"], sz["iters"], sg["ms"], sz["ms"], sg["guess_relres"]))
    # the network's own forward time at the size it runs on
    cells = tuple(guess["net_cells"])
    nc = cells[0] * cells[1] * cells[2]
    bin_ = torch.randn(nc, device=p.device)
    pin_ = torch.randn(nc, device=p.device)
    out = torch.empty_like(bin_)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    L.gn_forward(guess["handle"], cells, bin_, pin_, out)
    e0.record()
    for _ in range(5):
        L.gn_forward(guess["handle"], cells, bin_, pin_, out)
    e1.record()
    torch.cuda.synchronize()
    L.gn_destroy(guess["handle"])
    a = np.array(pairs)
    rec = {k: v_ for k, v_ in guess.items() if k != "handle"}
    rec.update({"guess_relres_mean": float(np.mean(rel)) if rel else None,
                "guess_relres_max": float(np.max(rel)) if rel else None, "rejected_steps": int(rej),
                "forward_ms": round(e0.elapsed_time(e1) / 5, 4),
                "same_state": {"steps": compare, "iters_guess": float(a[:, 0].mean()),
                               "iters_zero": float(a[:, 1].mean()),
                               "solve_ms_guess": float(a[:, 2].mean()), "solve_ms_zero": float(a[:, 3].mean())}})
    return rec


def run_gpu(args, rank, world):
    import torch
    from paper_2402_17913_gb300 import build, lib as L
    build.build()
    L.load()
    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    dev = torch.device("cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    guess = None

    if args.config in ("ns2d", "ns3d", "timing3d"):
        fe = args.stencil == "fe"
        opt, tol = None, TOL
        if args.config == "timing3d":
            wl = Timing3D(args.size, args.cycle)
            fe = True
            if args.cycle == "sawtooth":
                # a fixed 20 cycles: one inner solve of 20 cycles, with no
                # tolerance that could end it earlier
                opt = L.default_options(cycle=L.MG_CYCLE_SAWTOOTH, krylov=0, coarse_scale=0.5, max_inner=wl.iters,
                                        max_outer=1, inner_floor=1e-30)
                tol = 1e-30
        else:
            wl = NS2D(fe=fe) if args.config == "ns2d" else NS3D(fe=fe)
        solid_t = torch.from_numpy(wl.solid.astype(np.uint8)).to(dev)
        ns = L.ns_create(wl.dim, wl.cells, 1.0, solid_t, options=opt)
        if fe:
            L.ns_set_stencils(ns, L.NS_STENCIL_FE)
        mg = L.ns_pressure_handle(ns)
        if args.config == "timing3d":
            q = wl.initial_velocity()
        else:
            q = [a.astype(np.float32) for a in I.ns_initial_velocity(wl.cells, 0)]
        init = [a.copy() for a in q] + [np.zeros(wl.solid.shape, np.float32)]
        host = [torch.from_numpy(a.copy()).pin_memory() for a in init]
        fields = [t.to(dev) for t in host]
        u, v, p = fields[0], fields[1], fields[-1]
        w = fields[2] if wl.dim == 3 else None
        stats = []
        guess = None
        if args.config == "ns3d" and args.guess == "net":
            guess = train_guess(L, ns, wl, u, v, w, p, solid_t, args.train_steps, args.guess_level)
            # the timed run restarts from the initial state, so that it solves
            # the same sequence of problems as the zero-guess run
            for d, t in zip(host, fields):
                t.copy_(d)
            torch.cuda.synchronize()
        advance = args.advance if args.advance is not None else {"ns2d": 480, "ns3d": 180}.get(args.config, 0)
        for _ in range(advance):
            L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, tol, stats=False)
        torch.cuda.synchronize()
        wl.window = (advance + args.warmup + 1, advance + args.warmup + args.steps)

        def step():
            _, st = L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, tol)
            stats.append(st)

        def check():
            """One step from the seeded initial state (the state the oracle
            step starts from), fields as float32 numpy arrays."""
            for d, a in zip(fields, init):
                d.copy_(torch.from_numpy(a))
            status, st = L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, tol)
            torch.cuda.synchronize()
            return {"kind": "ns", "q": [t.cpu().numpy() for t in fields[:-1]], "p": fields[-1].cpu().numpy(),
                    "relres": st["relres"], "status": status}

        def e2e_step():
            for d, hsrc in zip(fields, host):
                d.copy_(hsrc, non_blocking=True)
            step()
            for d, hdst in zip(fields, host):
                hdst.copy_(d, non_blocking=True)
        io_bytes = sum(t.numel() * 4 for t in host)
        cleanup = lambda: L.ns_destroy(ns)  # noqa: E731
    elif args.config == "batched":
        wl = Batched(count=args.batch_count, rank=rank, world=world)
        masks = [torch.from_numpy(m.astype(np.uint8)).to(dev) for m in wl.solids]
        bh = L.mg_create_batched(wl.shapes, wl.spacings, (0, 0, 0, 0), masks)
        mg = None
        hb = [torch.from_numpy(r).pin_memory() for r in wl.rhs]
        hx = [torch.zeros_like(t).pin_memory() for t in hb]
        db = [t.to(dev) for t in hb]
        dx = [torch.zeros_like(t) for t in db]
        tuned = L.mg_tune_batched(bh, db, dx, TOL)
        stats = []

        def check():
            """The float32 results of the instances the oracle leg solves
            (the first 16 of the batch), from the last solve."""
            torch.cuda.synchronize()
            return {"kind": "batched", "x": {k: t.cpu().numpy() for k, t in zip(wl.index, dx) if k < 16}}

        def step():
            for t in dx:
                t.zero_()
            _, st = L.mg_solve_batched(bh, db, dx, TOL)
            stats.append({"iters": max(s_["iters"] for s_ in st), "relres": max(s_["relres"] for s_ in st),
                          "outer": max(s_["outer"] for s_ in st), "all": st})

        def e2e_step():
            for d, hsrc in zip(db, hb):
                d.copy_(hsrc, non_blocking=True)
            step()
            for d, hdst in zip(dx, hx):
                hdst.copy_(d, non_blocking=True)
        io_bytes = sum(t.numel() * 4 for t in hb)
        cleanup = lambda: L.mg_destroy_batched(bh)  # noqa: E731
    elif args.config == "advdiff":
        wl = AdvDiff(args.ad_size, args.cycle)
        if args.cycle == "sawtooth":
            opt = L.ad_default_options(cycle=L.MG_CYCLE_SAWTOOTH, pre=0, post=1, omega=1.0, coarse_scale=0.5,
                                       max_cycles=5000)
            ad_tol, ad_l1 = 0.0, 1e-5
        else:
            opt = L.ad_default_options()
            ad_tol, ad_l1 = TOL, 0.0
        hd = L.ad_create((wl.n, wl.n), wl.h, wl.dt, wl.nu, wl.u, wl.v, L.AD_UPWIND, opt)
        mg = None
        b_host = torch.from_numpy(wl.rhs()).pin_memory()
        x_host = torch.zeros_like(b_host).pin_memory()
        b = b_host.to(dev)
        x = torch.zeros_like(b)
        stats = []
        wl.levels, wl.kc = L.ad_num_levels(hd), L.ad_coarse_start(hd)

        def step():
            _, st = L.ad_solve(hd, b, x, rel_tol=ad_tol, l1_tol=ad_l1)
            stats.append(dict(st, iters=st["cycles"], outer=1))

        def e2e_step():
            b.copy_(b_host, non_blocking=True)
            step()
            x_host.copy_(x, non_blocking=True)
        io_bytes = b_host.numel() * 4
        check = None
        cleanup = lambda: L.ad_destroy(hd)  # noqa: E731
    else:
        shape = (256, 256) if args.config == "poisson2d" else (256, 256, 256)
        wl = Poisson(shape, args.prec, args.cycle)
        h = I.poisson_spacing(shape)
        opt = L.default_options(prec=PREC[args.prec])
        if args.cycle == "sawtooth":
            # the paper's cycle as a stationary solver; the re-discretised
            # coarse levels need the halved correction (the oracle's pin)
            opt = L.default_options(prec=PREC[args.prec], cycle=L.MG_CYCLE_SAWTOOTH, krylov=0, coarse_scale=0.5,
                                    max_inner=20000)
        mg = L.mg_create(wl.dim, tuple(reversed(shape)), h, (0,) * (2 * wl.dim), None, opt)
        b_host = torch.from_numpy(I.blob_rhs(shape, 0).astype(np.float32)).pin_memory()
        x_host = torch.zeros_like(b_host).pin_memory()
        b = b_host.to(dev)
        x = torch.zeros_like(b)
        stats = []

        def step():
            x.zero_()
            _, st = L.mg_solve(mg, b, x, TOL)
            stats.append(st)

        def check():
            """The float64 iterate and the float32 output of the last solve."""
            x64 = torch.zeros(shape, dtype=torch.float64, device=dev)
            L.mg_get_solution_f64(mg, x64)
            torch.cuda.synchronize()
            return {"kind": "poisson", "x64": x64.cpu().numpy(), "x32": x.cpu().numpy(),
                    "relres": stats[-1]["relres"] if stats else None}

        def e2e_step():
            b.copy_(b_host, non_blocking=True)
            step()
            x_host.copy_(x, non_blocking=True)
        io_bytes = b_host.numel() * 4
        cleanup = lambda: L.mg_destroy(mg)  # noqa: E731

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats.clear()
    gn_launches0 = L.gn_kernel_launches()
    dist_barrier(world)
    # ---- timed: device-resident inputs, L2 flushed between steps
    launches0 = L.mg_kernel_launches(mg) if mg else (L.ad_kernel_launches(hd) if args.config == "advdiff" else 0)
    cp, cf, cpath = clocks_sampler()
    times = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    # an NVTX range around the timed steps: a profiler capture can take
    # exactly their launches (ncu --nvtx --nvtx-include "timed/")
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        step()
        ev[i][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = clocks_summary(cp, cf, cpath)
    times = [a.elapsed_time(b) for a, b in ev]
    # the batched solve is one persistent kernel per solve (one graph launch)
    launches = (L.mg_kernel_launches(mg) - launches0) if mg else args.steps
    if args.config == "advdiff":
        launches = L.ad_kernel_launches(hd) - launches0
    launches += L.gn_kernel_launches() - gn_launches0
    step_stats = list(stats)
    total_ms = dist_max(sum(times), world)
    if args.only_timed:
        cleanup()
        return {"metric": METRIC, "value": wl.units * args.steps * world / (total_ms * 1e-3), "unit": UNIT,
                "steps": args.steps, "only_timed": True, "gpu_launches": int(launches)}, wl
    # ---- end to end: host buffers, copies inside the timed region
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        e2e_step()
        t1.record()
        torch.cuda.synchronize()
        e2e_ms.append(t0.elapsed_time(t1))
    e2e_total = dist_max(sum(e2e_ms), world)
    check_data = check() if (check is not None and rank == 0) else None
    guess_rec = guess_report(L, guess, step_stats, ns, wl, u, v, w, p) if guess else None
    peak, peak_kind = measured_peak()
    if args.config == "batched":
        # the whole solve is one persistent kernel: its algorithmic bytes are
        # the per-cell bytes of each CG iteration and refinement pass of every
        # instance (BATCH_ITER_BYTES, OUTER_BYTES), over the event-timed solve
        cleanup()
        last = step_stats[-1]["all"]
        algo = sum((st["iters"] * BATCH_ITER_BYTES + (st["outer"] + 1) * OUTER_BYTES) * n * n
                   for st, (n, _) in zip(last, wl.shapes))
        ms_solve = total_ms / args.steps
        achieved = algo / (ms_solve * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_batched (persistent)", "achieved": round(achieved, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                    "traffic": recorded_traffic(wl.name, "k_batched"), "algorithmic_bytes_per_launch": algo,
                    "avg_launch_us": round(ms_solve * 1e3, 2), "share_of_step": 1.0,
                    "autotuned": {"tile": [tuned[0], tuned[1]], "sweeps": tuned[2]}}
    elif args.config == "advdiff":
        # the whole solve: algorithmic bytes of one cycle over the
        # event-timed solve (level 0: residual 16 B per node - b, float64 x,
        # r -; down leg 9 B; up leg 25 B - b, x, 1/4 e, float64 x read and
        # written -; each tile level below: 22 B per node; the single block's
        # levels stay on chip)
        cleanup()
        n0 = wl.units
        per_cycle = 50 * n0 + sum(22 * (n0 >> (2 * k)) for k in range(1, wl.kc))
        cyc = statistics.mean(st["cycles"] for st in step_stats)
        ms_solve = total_ms / args.steps
        achieved = per_cycle * cyc / (ms_solve * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": "whole solve (k_ad_resid, k_ad_down, k_ad_coarse, k_ad_up)",
                    "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": None,
                    "algorithmic_bytes_per_cycle": per_cycle, "cycles_per_solve": cyc,
                    "levels": wl.levels, "single_block_from_level": wl.kc,
                    "avg_cycle_us": round(ms_solve * 1e3 / max(cyc, 1), 2)}
    else:
        # ---- profiled pass: per-kernel-class event times (graph off)
        L.mg_profile_enable(mg, True)
        L.mg_profile_read(mg, reset=True)
        nprof = min(args.steps, 5)
        for i in range(nprof):
            flush.fill_(float(i))
            step()
        prof = L.mg_profile_read(mg, reset=True)
        L.mg_profile_enable(mg, False)
        cleanup()
        tot_prof = sum(ms for ms, _ in prof.values()) or 1.0
        dom = max(KERNEL_CLASSES + ("cluster_pcg",), key=lambda k: prof[k][0])
        ms_dom, n_dom = prof[dom]
        is_ns = args.config in ("ns2d", "ns3d", "timing3d")
        ncell = int(np.prod(wl.cells)) if is_ns else wl.units
        prec_b = "fp32" if is_ns else args.prec
        if dom == "cluster_pcg":
            # one launch runs an inner solve's CG iterations: their algorithmic
            # bytes as if each pass moved its finest arrays once
            its = statistics.mean(st["iters"] for st in step_stats) * nprof / max(n_dom, 1)
            per_cell = its * sum(algo_bytes_per_cell(k, wl.dim, prec_b, masked=is_ns)
                                 for k in ("down_fine", "up_fine", "p_update", "xr_update"))
        else:
            per_cell = algo_bytes_per_cell(dom, wl.dim, prec_b, masked=is_ns)
        algo = per_cell * ncell
        us = ms_dom / max(n_dom, 1) * 1e3
        achieved = algo / (us * 1e-6) / 1e9
        roofline = {"kernel": dom, "achieved": round(achieved, 1), "unit": "GB/s",
                    "algorithmic_bytes_per_cell": per_cell, "algorithmic_bytes_per_launch": algo,
                    "avg_launch_us": round(us, 2), "share_of_step": round(ms_dom / tot_prof, 3),
                    "class_shares": {k: round(v[0] / tot_prof, 3) for k, v in prof.items() if v[1]}}
        l2_size = torch.cuda.get_device_properties(dev).L2_cache_size
        if ncell * LIVE_BYTES_PER_CELL < l2_size:
            # the solve's arrays stay in L2 between launches (DRAM sees almost
            # none of the traffic): the roof is L2, measured live
            l2 = l2_read_peak(L, dev, l2_size)
            roofline.update(bound="l2", peak=round(l2, 1), peak_source="measured live (mg_probe_l2_read)",
                            frac=round(achieved / l2, 4), traffic=None,
                            hbm={"peak": peak, "peak_source": peak_kind, "frac": round(achieved / peak, 4)})
        else:
            roofline.update(bound="hbm", peak=peak, peak_source=peak_kind, frac=round(achieved / peak, 4),
                            traffic=recorded_traffic(wl.name, dom))
    # whole-job rate: replicas each solve their own step (weak scaling); the
    # batched workload is one batch split over the ranks (strong scaling)
    split = getattr(wl, "job_units", None)
    value = job_rate(wl.units, args.steps, world, total_ms) if split is None else \
        split * args.steps / (total_ms * 1e-3)
    e2e_value = (wl.units * args.steps * world if split is None else split * args.steps) / (e2e_total * 1e-3)
    its = [s["iters"] for s in step_stats]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak" if split is None else "strong", "vs_baseline": None,
        "dtype": "f32" if args.prec == "fp32" else args.prec,
        "data": "synthetic", "config": dict(wl.config(), parallelism="replicas" if world > 1 else "single"),
        "clocks": clocks, "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "roofline": roofline,
        "guess": guess_rec,
        "solve": {"cg_iters_mean": statistics.mean(its) if its else None,
                  "relres_max": max(s["relres"] for s in step_stats) if step_stats else None,
                  "outer_mean": statistics.mean(s["outer"] for s in step_stats) if step_stats else None},
    }
    if args.config == "advdiff":
        out["solve"].update(cycles_mean=out["solve"].pop("cg_iters_mean"),
                            l1_first=step_stats[-1]["l1_first"], l1_last=step_stats[-1]["l1_last"])
        if args.cycle == "sawtooth":
            out["metric"] = AD_L1_METRIC
            out["e2e"]["unit"] = UNIT
    if args.config == "timing3d":
        # the paper's metric: seconds for five time steps of 20 iterations
        t4 = wl.paper_s.get(wl.n, (None, None))[0]
        five = 5 * total_ms / args.steps / 1e3
        out.update(metric=TIMING_METRIC, value=five, unit="s", higher_is_better=False,
                   vs_baseline=(five / t4 if t4 and args.cycle == "sawtooth" else None), unknowns_per_s=value)
        out["e2e"] = dict(out["e2e"], value=5 * e2e_total / args.steps / 1e3, unit="s")
        out["solve"]["relres_per_step"] = [s["relres"] for s in step_stats]
    if args.config == "poisson3d" and args.prec == "fp32" and args.cycle == "v":
        # the same solve with FP16 / BF16 level storage, against this line's
        # plain float32 form
        out["mixed_precision"] = {}
        for prec in ("fp16", "bf16"):
            rec = time_poisson(L, dev, flush, wl.shape, prec, args.steps, args.warmup)
            rec["vs_fp32"] = round(rec["value"] / value, 4)
            out["mixed_precision"][prec] = rec
    out["_check"] = check_data
    return out, wl


def time_poisson(L, dev, flush, shape, prec, steps, warmup):
    """Solves of the blob workload to relres 1e-6 with level storage `prec`:
    unknowns/s over `steps` event-timed solves (L2 flushed between them),
    iterations, relres, and the up_fine class's fraction of the measured
    copy bandwidth from a profiled pass."""
    import torch
    h = I.poisson_spacing(shape)
    mg = L.mg_create(len(shape), tuple(reversed(shape)), h, (0,) * (2 * len(shape)), None,
                     L.default_options(prec=PREC[prec]))
    try:
        b = torch.from_numpy(I.blob_rhs(shape, 0).astype(np.float32)).to(dev)
        x = torch.zeros_like(b)
        stats = []
        for _ in range(warmup):
            x.zero_()
            L.mg_solve(mg, b, x, TOL)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(float(i))
            x.zero_()
            ev[i][0].record()
            stats.append(L.mg_solve(mg, b, x, TOL)[1])
            ev[i][1].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in ev) / steps
        L.mg_profile_enable(mg, True)
        L.mg_profile_read(mg, reset=True)
        for i in range(min(steps, 5)):
            flush.fill_(float(i))
            x.zero_()
            L.mg_solve(mg, b, x, TOL)
        prof = L.mg_profile_read(mg, reset=True)
        L.mg_profile_enable(mg, False)
    finally:
        L.mg_destroy(mg)
    units = int(np.prod(shape))
    per_cell = algo_bytes_per_cell("up_fine", len(shape), prec)
    ms_up, n_up = prof["up_fine"]
    achieved = per_cell * units / (ms_up / max(n_up, 1) * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    return {"value": units / (ms * 1e-3), "ms_per_step": round(ms, 4),
            "cg_iters_mean": statistics.mean(s["iters"] for s in stats),
            "relres_max": max(s["relres"] for s in stats),
            "up_fine": {"algorithmic_bytes_per_cell": per_cell, "achieved": round(achieved, 1),
                        "frac": round(achieved / peak, 4), "peak": peak, "peak_source": peak_kind}}


def oracle_step_time(wl, budget_s=30.0, max_steps=3):
    """Time the FP64 oracle (as it stands) on a bounded sample of workload
    `wl`; returns (unknowns/s, sample description, steps timed)."""
    from oracle import ns as N
    from oracle import poisson as P
    t_total, steps, units = 0.0, 0, 0
    if isinstance(wl, (NS2D, NS3D, Timing3D)):
        g = N.MacGrid(wl.cells, 1.0, wl.solid)
        hier = P.build_hierarchy(g.shape, (1.0,) * wl.dim, g.p_bc, wl.solid)
        if isinstance(wl, Timing3D) and wl.cycle == "sawtooth":
            q = [a.astype(np.float64) for a in wl.initial_velocity()]
            mg = P.Multigrid(hier, post=2, s=0.5, cycle='sawtooth')
            solve = lambda b: mg.stationary(b, wl.iters)[0]  # noqa: E731
        elif isinstance(wl, Timing3D):
            q = [a.astype(np.float64) for a in wl.initial_velocity()]
            mg = P.Multigrid(hier, s=1.0)
            solve = lambda b: P.pcg_ir(mg, b, tol=TOL)[0]  # noqa: E731
        else:
            mg = P.Multigrid(hier, s=1.0)
            q = I.ns_initial_velocity(wl.cells, 0)
            solve = lambda b: P.pcg_ir(mg, b, tol=TOL)[0]  # noqa: E731
        p = np.zeros(g.shape)
        while steps < max_steps and t_total < budget_s:
            t0 = time.perf_counter()
            q, p, _, _, _ = N.ns_step(g, q, p, wl.dt, wl.nu, wl.uin, solve=solve, fe=wl.fe)
            t_total += time.perf_counter() - t0
            steps += 1
            units += wl.units
        sample = "%d oracle step(s) of the %s projection workload (%s)" % (
            steps, "x".join(map(str, wl.cells)),
            "20 sawtooth cycles" if isinstance(wl, Timing3D) and wl.cycle == "sawtooth" else "pressure solve to 1e-6")
    elif isinstance(wl, AdvDiff):
        from oracle import advdiff as AD
        hier = AD.build_hierarchy(wl.shape, wl.h, wl.dt, wl.nu, wl.u, wl.v, 'upwind', 'rediscretise')
        if wl.cycle == "sawtooth":
            mg = AD.ADMultigrid(hier, 'sawtooth', 0, 1, 1.0, 0.5)
            kw = dict(tol=0.0, l1_tol=1e-5, max_cycles=5000)
        else:
            mg = AD.ADMultigrid(hier, 'V', 2, 2, 2.0 / 3.0, 1.0)
            kw = dict(tol=TOL)
        b = wl.rhs().astype(np.float64)
        while steps < max_steps and t_total < budget_s:
            t0 = time.perf_counter()
            mg.solve(b, **kw)
            t_total += time.perf_counter() - t0
            steps += 1
            units += wl.units
        sample = "%d oracle solve(s) of the %d^2 advection-diffusion step" % (steps, wl.n)
    elif isinstance(wl, Batched):
        for k in range(len(wl.shapes)):
            if steps >= max_steps or t_total >= budget_s:
                break
            n = wl.shapes[k][0]
            hier = P.build_hierarchy((n, n), wl.spacings[k], (0, 0, 0, 0), wl.solids[k])
            mg = P.Multigrid(hier, s=1.0)
            b = wl.rhs[k].astype(np.float64)
            t0 = time.perf_counter()
            P.pcg_ir(mg, b, tol=TOL)
            t_total += time.perf_counter() - t0
            steps += 1
            units += int((~wl.solids[k]).sum())
        sample = "the first %d instances of the batch, each solved by the oracle to 1e-6" % steps
    else:
        shape = wl.shape
        h = I.poisson_spacing(shape)
        hier = P.build_hierarchy(shape, h, (0,) * (2 * len(shape)))
        mg = P.Multigrid(hier, s=1.0)
        b = I.blob_rhs(shape, 0).astype(np.float32).astype(np.float64)
        while steps < max_steps and t_total < budget_s:
            t0 = time.perf_counter()
            P.pcg_ir(mg, b, tol=TOL)
            t_total += time.perf_counter() - t0
            steps += 1
            units += wl.units
        sample = "%d oracle solve(s) of the %s workload to 1e-6" % (steps, "x".join(map(str, shape)))
    return units / t_total, sample, steps


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(units_per_step, steps, world, max_ms):
    """Whole-job throughput of `world` replicas that each did `steps` steps
    of `units_per_step` unknowns, timed by the slowest rank (max_ms)."""
    return units_per_step * steps * world / (max_ms * 1e-3)


def dist_max(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launch_ranks(n):
    """`--gpus N` without a launcher: run this command under
    torch.distributed.run with N ranks on this node (127.0.0.1) and return
    its exit code."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(n),
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    world_env = os.environ.get("WORLD_SIZE")
    if world_env is None and args.gpus > 1:
        sys.exit(launch_ranks(args.gpus))
    if int(world_env or "1") != args.gpus:
        sys.exit("bench.py: --gpus %d but WORLD_SIZE=%s; launch one rank per GPU" % (args.gpus, world_env))
    rank, world = dist_init()
    if args.impl == "reference":
        if rank != 0:
            return
        # each reference step is one oracle step of a bounded sample of the
        # workload (same structure, fewer cells), so the run ends in minutes
        fe = args.stencil == "fe"
        samples = {"ns2d": lambda: NS2D(scale=4, fe=fe), "ns3d": lambda: NS3D(scale=4, fe=fe),
                   "poisson2d": lambda: Poisson((256, 256), args.prec),
                   "poisson3d": lambda: Poisson((64, 64, 64), args.prec), "batched": lambda: Batched(limit=16),
                   "timing3d": lambda: Timing3D(args.size, args.cycle, scale=args.size // 32),
                   "advdiff": lambda: AdvDiff(min(args.ad_size, 512), args.cycle)}
        wl = samples[args.config]()
        t0 = time.perf_counter()
        rate, sample, n = oracle_step_time(wl, budget_s=1e9, max_steps=args.warmup + args.steps)
        cores = 1
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(wl.config(), sample={
                    "ns2d": "quarter-resolution copy (512x256 cells, 16-cell block, Re kept at 100)",
                    "ns3d": "quarter-resolution copy (64x32x32 cells, 8-cell cube, Re kept at 100)",
                    "poisson3d": "64^3 copy of the blob workload",
                    "batched": "the first 16 instances of the batch",
                    "timing3d": "32^3 copy (cube and Re scaled alike); seconds scaled to the full size by cells",
                    "advdiff": "the step itself up to 512^2 nodes, else a 512^2 copy"}.get(
                        args.config, "the workload itself")),
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        if args.config == "advdiff" and args.cycle == "sawtooth":
            line["metric"] = AD_L1_METRIC
        if args.config == "timing3d":
            full = Timing3D(args.size, args.cycle)
            secs = 5 * full.units / rate
            line.update(metric=TIMING_METRIC, value=secs, unit="s", higher_is_better=False, unknowns_per_s=rate)
            line["cpu_baseline"] = dict(line["cpu_baseline"], value=secs, unit="s")
            line["e2e"] = dict(line["e2e"], value=secs, unit="s")
        print(json.dumps(line))
        return
    # the oracle's answer to the GPU line's own problem, computed in a spawn
    # worker (started before this process touches the GPU) while the GPU runs
    pool = fut = None
    want_check = (rank == 0 and world == 1 and not args.only_timed and not args.no_cpu_baseline
                  and args.config in ("poisson2d", "poisson3d", "ns2d", "ns3d") and args.cycle == "v")
    if want_check:
        import concurrent.futures
        import multiprocessing
        # the worker's BLAS and OpenMP pools held to a few threads, so that it
        # leaves the host cores that drive the GPU alone (spawned children
        # read these at start)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({k: "2" for k in saved})
        try:
            pool = concurrent.futures.ProcessPoolExecutor(1, mp_context=multiprocessing.get_context("spawn"))
            fut = pool.submit(oracle_reference, args.config, args.stencil == "fe")
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    out, wl = run_gpu(args, rank, world)
    check = out.pop("_check", None)
    if rank == 0:
        ref = None
        if fut is not None:
            # wait for the worker before the CPU baseline is timed, so that
            # the two do not share the host cores
            ref = fut.result()
            pool.shutdown()
        if not args.no_cpu_baseline and world == 1 and not args.only_timed:
            spec = sample_spec(args)
            rate, sample, n = oracle_step_time(cpu_sample(spec), budget_s=25.0, max_steps=spec["max_steps"])
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
            agg, procs = oracle_all_cores(spec)
            out["cpu_baseline"]["all_cores"] = {
                "value": agg, "unit": UNIT, "cores": procs, "kind": "oracle",
                "sample": "%d copies of the same sample at once, one process per core" % procs}
            if args.config == "timing3d":
                # the line's unit: seconds for five steps, scaled by cells
                out["cpu_baseline"].update(value=5 * wl.units / rate, unit="s",
                                           sample=sample + "; seconds scaled to the full size by cells")
                out["cpu_baseline"]["all_cores"].update(value=5 * wl.units / agg, unit="s")
        if fut is not None:
            out["oracle_check"] = compare_with_oracle(args.config, check, ref, args.stencil == "fe")
        print(json.dumps(out))


def sample_spec(args):
    """The bounded sample the CPU baseline times (picklable)."""
    return {"config": args.config, "prec": args.prec, "size": args.size, "cycle": args.cycle,
            "ad_size": args.ad_size, "fe": args.stencil == "fe",
            "max_steps": {"poisson2d": 5, "batched": 64}.get(args.config, 1)}


def cpu_sample(spec):
    """Workload of the CPU baseline: the GPU line's own workload, or (3D, and
    the large advection-diffusion grids) a smaller copy the oracle finishes
    in seconds."""
    c, fe = spec["config"], spec["fe"]
    if c == "ns2d":
        return NS2D(fe=fe)
    if c == "ns3d":
        return NS3D(scale=2, fe=fe)
    if c == "timing3d":
        return Timing3D(spec["size"], spec["cycle"], scale=max(1, spec["size"] // 64))
    if c == "advdiff":
        return AdvDiff(min(spec["ad_size"], 512), spec["cycle"])
    if c == "poisson3d":
        return Poisson((128, 128, 128), spec["prec"])
    if c == "poisson2d":
        return Poisson((256, 256), spec["prec"], spec["cycle"])
    return Batched()


def _oracle_sample_worker(spec, start_at):
    wl = cpu_sample(spec)
    while time.time() < start_at:  # every process starts its timing together
        time.sleep(0.01)
    t0 = time.time()
    rate, _, n = oracle_step_time(wl, budget_s=1.0, max_steps=1)
    return rate * (time.time() - t0), t0, time.time()


def oracle_all_cores(spec):
    """The oracle on every host core at once: one process per core, each
    timing one step of the same sample; aggregate unknowns/s = all units /
    the span from the first start to the last end."""
    import concurrent.futures
    import multiprocessing
    procs = min(os.cpu_count() or 1, 16)
    # one core per process: the BLAS and OpenMP pools of each child to one
    # thread (spawned children read these at start)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        with concurrent.futures.ProcessPoolExecutor(procs, mp_context=multiprocessing.get_context("spawn")) as ex:
            start_at = time.time() + 20.0 + 0.5 * procs  # time to spawn and build the samples
            res = list(ex.map(_oracle_sample_worker, [spec] * procs, [start_at] * procs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return units / span, procs


def oracle_reference(config, fe=False):
    """The FP64 oracle's answer to the problem the GPU line also solves:
    the Poisson blob workload solved by the oracle's MG-PCG with refinement
    to relres 1e-6 (the same stopping rule), or one projection step from the
    seeded initial state with the pressure solved to relres 1e-12."""
    from oracle import ns as N
    from oracle import poisson as P
    if config in ("poisson2d", "poisson3d"):
        shape = (256, 256) if config == "poisson2d" else (256, 256, 256)
        b = I.blob_rhs(shape, 0).astype(np.float32).astype(np.float64)
        mg = P.Multigrid(P.build_hierarchy(shape, I.poisson_spacing(shape), (0,) * (2 * len(shape))), s=1.0)
        x, hist, inner = P.pcg_ir(mg, b, tol=TOL)
        return {"x": x, "relres": hist[-1], "iters": inner}
    wl = NS2D(fe=fe) if config == "ns2d" else NS3D(fe=fe)
    q = [a.astype(np.float32).astype(np.float64) for a in I.ns_initial_velocity(wl.cells, 0)]
    g = N.MacGrid(wl.cells, 1.0, wl.solid)
    qn, pn, _, _, _ = N.ns_step(g, q, np.zeros(wl.solid.shape), wl.dt, wl.nu, wl.uin, fe=fe)
    return {"q": qn, "p": pn}


def compare_with_oracle(config, gpu, ref, fe=False):
    """Error of the GPU result against the oracle's, per result."""
    from oracle import poisson as P
    if gpu is None or ref is None:
        return None
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))  # noqa: E731
    if gpu["kind"] == "poisson":
        shape = (256, 256) if config == "poisson2d" else (256, 256, 256)
        lv = P.Level(shape, I.poisson_spacing(shape), (0,) * (2 * len(shape)))
        b = I.blob_rhs(shape, 0).astype(np.float32).astype(np.float64)
        return {"what": "the timed solve's result vs the oracle's MG-PCG solve to the same relres 1e-6",
                "relres_gpu_float64_iterate": P.relres(lv, b, gpu["x64"]),
                "relres_gpu_float32_output": P.relres(lv, b, gpu["x32"].astype(np.float64)),
                "relerr_float64_iterate": rel(gpu["x64"], ref["x"]), "relerr_float32_output":
                rel(gpu["x32"].astype(np.float64), ref["x"]),
                "oracle_relres": ref["relres"], "oracle_cg_iters": ref["iters"]}
    out = {"what": "one step from the seeded initial state vs the oracle's step (pressure solved to 1e-12)",
           "relres_gpu": gpu["relres"]}
    for c, name in enumerate("uvw"[:len(gpu["q"])]):
        out["relerr_" + name] = rel(gpu["q"][c].astype(np.float64), ref["q"][c])
    out["relerr_p"] = rel(gpu["p"].astype(np.float64), ref["p"])
    return out


if __name__ == "__main__":
    main()
