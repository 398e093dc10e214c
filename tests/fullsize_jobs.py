"""Oracle runs for the full-size parity tests (tests/test_gpu_fullsize.py).

Each function rebuilds its workload from the seeded generators of
``paper_2402_17913_gb300.inputs`` (the same recipe the benchmark uses) and
runs only ``oracle/`` code on it, so no expected value depends on the GPU
path.  They run in worker processes started with ``spawn`` (the oracle runs
take minutes at these sizes; several run side by side while the GPU tests
proceed).  Not collected by pytest (no ``test_`` prefix).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ns as N  # noqa: E402
from oracle import poisson as P  # noqa: E402
from paper_2402_17913_gb300 import inputs as I  # noqa: E402

# the 3D pressure-Poisson workload: 256^3 cells, 8 blobs (seed 0), zero Dirichlet
POISSON3D = (256, 256, 256)
# the 2D projection step: 2048 x 1024 cells, a 64-cell block at (512, 512)
NS2D = dict(cells=(2048, 1024), block=64, centre=(512, 512), nu=0.64)
# the 3D projection step: 256 x 128 x 128 cells, a 32-cell cube at (64, 64, 64)
NS3D = dict(cells=(256, 128, 128), block=32, centre=(64, 64, 64), nu=0.32)
DT, U_IN = 0.1, 1.0
# the batched workload: sides and solid fractions from seed 1234
BATCH_SEED, BATCH_COUNT = 1234, 1024
X_STAR_TOL = 1e-11


def poisson3d_rhs():
    return I.blob_rhs(POISSON3D, 0).astype(np.float32)


def poisson3d_x_star():
    """x* = A_h^{-1} b of the 256^3 workload by the oracle's MG-PCG to relres
    1e-11 (FP64)."""
    shape = POISSON3D
    b = poisson3d_rhs().astype(np.float64)
    return P.solve_reference(shape, I.poisson_spacing(shape), (0,) * 6, b, None, tol=X_STAR_TOL, s=1.0)


def ns_case(spec):
    cells = spec["cells"]
    solid = I.block_mask(cells, spec["centre"], spec["block"])
    q = [a.astype(np.float32) for a in I.ns_initial_velocity(cells, 0)]
    p = np.zeros(solid.shape, np.float32)
    return cells, solid, q, p


def ns_oracle_step(name):
    """One oracle projection step (pressure solve to relres 1e-12) from the
    seeded initial state of the 2D or 3D flow workload; returns the new
    velocity components, pressure, and the divergence of q*."""
    spec = NS2D if name == "ns2d" else NS3D
    cells, solid, q, p = ns_case(spec)
    g = N.MacGrid(cells, 1.0, solid)
    qn, pn, dp, qs, b = N.ns_step(g, [a.astype(np.float64) for a in q], p.astype(np.float64), DT, spec["nu"], U_IN)
    dstar = float(np.linalg.norm(g.divergence(qs)[~solid]))
    return {"q": qn, "p": pn, "div_star": dstar}


def batch_subset(per_side=2, scan=40):
    """Instances of the batched workload (in the workload's own draw order,
    so the masks are the ones the benchmark solves): for every side in
    {64, 128, 256, 512} the first ``per_side`` instances of that side and the
    one with the largest solid fraction among the first ``scan`` instances.
    Returns a list of (index, n, solid, rhs float32)."""
    sides, fracs, rng = I.batched_sides(BATCH_COUNT, BATCH_SEED)
    chosen, seen, best = {}, {}, {}
    for k in range(scan):
        n, f = sides[k], fracs[k]
        solid = I.random_solid_mask((n, n), rng, f)
        seen[n] = seen.get(n, 0) + 1
        if seen[n] <= per_side:
            chosen[k] = (n, solid)
        if n not in best or f > best[n][0]:
            best[n] = (f, k, solid)
    for n, (f, k, solid) in best.items():
        chosen[k] = (n, solid)
    out = []
    for k in sorted(chosen):
        n, solid = chosen[k]
        out.append((k, n, solid, I.blob_rhs((n, n), k, solid=solid).astype(np.float32)))
    return out


def batch_x_star():
    """x* of every instance of ``batch_subset()`` (oracle MG-PCG to 1e-12)."""
    res = []
    for k, n, solid, b in batch_subset():
        h = (1.0 / (n + 1),) * 2
        res.append(P.solve_reference((n, n), h, (0, 0, 0, 0), b.astype(np.float64), solid, tol=1e-12, s=1.0))
    return res
