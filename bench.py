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

# Algorithmic bytes per fine-grid cell of one launch of each kernel class
# (float32 storage, the method's own minimum: each array read or written
# once per launch; masked levels read one cell byte more).  Only classes
# that dominate a step are listed.
# Batched solve: bytes per fine cell of one CG iteration (the four fine
# passes above, plus one cell byte in three of them, plus about a third more
# for the coarser levels) and of one float-float refinement pass.
BATCH_ITER_BYTES = 72
OUTER_BYTES = 28

ALGO_BYTES_PER_CELL = {
    "down_fine": 4 + 4 + 1,          # read b (= CG residual); write x, coarse b (1/4)
    "up_fine": 4 + 4 + 1 + 4,        # read b, x, coarse e (1/4); write z
    "p_update": 4 + 4 + 4 + 4,       # read z, p_old; write p, Ap
    "xr_update": 4 + 4 + 8 + 8,      # read p, Ap; read+write d, r
    "outer": 4 + 8 + 4 + 8 + 4,      # read b, x64, d; write x64, r'
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="ns2d",
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
                "momentum_filters": FILTERS[self.fe], "l2": "256 MiB buffer written between timed steps"}


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
                "l2": "256 MiB buffer written between timed steps"}


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


class Batched:
    """1024 independent square instances, sides uniform in {64, 128, 256,
    512} (seed 1234), random rectangle solids covering U(0, 0.1) of the
    cells (flood-filled), 8-blob right-hand sides (seed = instance index),
    zero Dirichlet faces.  Under several ranks each rank solves its own
    1024 instances (sides seed 1234 + rank, right-hand-side seeds offset by
    rank x 1024): the batch shards by instances with no collective; rank 0
    has the single-GPU workload."""
    name = "batched_1024"
    dim = 2

    def __init__(self, count=1024, seed=1234, limit=None, rank=0):
        self.rank = rank
        sides, fracs, rng = I.batched_sides(count, seed + rank)
        self.shapes, self.spacings, self.solids, self.rhs = [], [], [], []
        for k, (n, f) in enumerate(zip(sides, fracs)):
            if limit is not None and k >= limit:
                break
            solid = I.random_solid_mask((n, n), rng, f)
            self.shapes.append((n, n))
            self.spacings.append((1.0 / (n + 1), 1.0 / (n + 1)))
            self.solids.append(solid)
            self.rhs.append(I.blob_rhs((n, n), k + rank * count, solid=solid).astype(np.float32))
        self.units = int(sum((~s).sum() for s in self.solids))
        self.cells = int(sum(n * n for n, _ in self.shapes))

    def config(self):
        return {"workload": "batched 2D Poisson, %d instances of sides {64,128,256,512}, random solids"
                % len(self.shapes), "cells": self.cells, "solve_rel_tol": TOL, "unknowns_per_step": self.units,
                "l2": "inputs (%.1f GB) larger than L2" % (self.cells * 60 / 1e9),
                "sharding": "each rank solves its own instances (seeds offset by rank), no collective"}


PREC = {"fp32": 0, "fp16": 1, "bf16": 2}


# ---------------------------------------------------------------------------
def clocks_sampler():
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
            "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The translation unit of the dominant kernel of each workload with a
# committed traffic summary; its hash also covers the headers it includes.
TRAFFIC_TU = {"ns2d_block_2048x1024": "mg_stream2d.cu", "poisson3d_256x256x256_fp32": "mg_rows3d.cu",
              "ns3d_cube_256x128x128": "mg_rows3d.cu"}
KERNEL_HEADERS = ["mg_kernels.cuh", "launch.h", "npmg_internal.cuh"]


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
        host = [torch.from_numpy(a).pin_memory() for a in q + [np.zeros(wl.solid.shape, np.float32)]]
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

        def step():
            _, st = L.ns_step(ns, u, v, w, p, wl.dt, wl.nu, wl.uin, tol)
            stats.append(st)

        def e2e_step():
            for d, hsrc in zip(fields, host):
                d.copy_(hsrc, non_blocking=True)
            step()
            for d, hdst in zip(fields, host):
                hdst.copy_(d, non_blocking=True)
        io_bytes = sum(t.numel() * 4 for t in host)
        cleanup = lambda: L.ns_destroy(ns)  # noqa: E731
    elif args.config == "batched":
        wl = Batched(rank=rank)
        masks = [torch.from_numpy(m.astype(np.uint8)).to(dev) for m in wl.solids]
        bh = L.mg_create_batched(wl.shapes, wl.spacings, (0, 0, 0, 0), masks)
        mg = None
        hb = [torch.from_numpy(r).pin_memory() for r in wl.rhs]
        hx = [torch.zeros_like(t).pin_memory() for t in hb]
        db = [t.to(dev) for t in hb]
        dx = [torch.zeros_like(t) for t in db]
        tuned = L.mg_tune_batched(bh, db, dx, TOL)
        stats = []

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
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        step()
        ev[i][1].record()
    torch.cuda.synchronize()
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
        dom = max(ALGO_BYTES_PER_CELL, key=lambda k: prof[k][0])
        ms_dom, n_dom = prof[dom]
        is_ns = args.config in ("ns2d", "ns3d", "timing3d")
        ncell = int(np.prod(wl.cells)) if is_ns else wl.units
        per_cell = ALGO_BYTES_PER_CELL[dom] + (1 if is_ns and dom != "xr_update" else 0)
        if args.prec != "fp32" and not is_ns:
            per_cell = per_cell / 2.0 if dom not in ("outer",) else 8 + 4 + 2 + 8 + 2
        algo = per_cell * ncell
        achieved = algo / (ms_dom / max(n_dom, 1) * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                    "traffic": recorded_traffic(wl.name, dom), "algorithmic_bytes_per_launch": algo,
                    "avg_launch_us": round(ms_dom / max(n_dom, 1) * 1e3, 2),
                    "share_of_step": round(ms_dom / tot_prof, 3),
                    "class_shares": {k: round(v[0] / tot_prof, 3) for k, v in prof.items() if v[1]}}
    value = job_rate(wl.units, args.steps, world, total_ms)
    its = [s["iters"] for s in step_stats]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else args.prec,
        "data": "synthetic", "config": dict(wl.config(), parallelism="replicas" if world > 1 else "single"),
        "clocks": clocks, "gpu_launches": int(launches),
        "e2e": {"value": wl.units * args.steps * world / (e2e_total * 1e-3), "unit": UNIT,
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
    return out, wl


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


def main():
    args = parse()
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
    out, wl = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1 and not args.only_timed:
            ms = {"poisson2d": 5, "batched": 64}.get(args.config, 1)
            # 3D: the full-size oracle step takes minutes; time a smaller copy
            cpu_wl = {"ns3d": lambda: NS3D(scale=2, fe=wl.fe),
                      "timing3d": lambda: Timing3D(args.size, args.cycle, scale=max(1, args.size // 64)),
                      "advdiff": lambda: AdvDiff(min(args.ad_size, 512), args.cycle),
                      "poisson3d": lambda: Poisson((128, 128, 128), args.prec)}.get(
                args.config, lambda: wl)()
            rate, sample, n = oracle_step_time(cpu_wl, budget_s=25.0, max_steps=ms)
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
            if args.config == "timing3d":
                # the line's unit: seconds for five steps, scaled by cells
                out["cpu_baseline"].update(value=5 * wl.units / rate, unit="s",
                                           sample=sample + "; seconds scaled to the full size by cells")
        print(json.dumps(out))


if __name__ == "__main__":
    main()
