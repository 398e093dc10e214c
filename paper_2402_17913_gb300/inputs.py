"""Seeded synthetic inputs for the pressure-Poisson and projection-step
workloads.

This module holds no arithmetic of the solver: it only draws right-hand
sides, solid masks and initial velocity fields from fixed numpy PCG64 seeds,
so that the GPU library's tests and benchmark and the CPU oracle see the same
inputs.  Every generator returns float64 arrays; callers that feed the GPU
round them to float32 and give the oracle the same rounded values.

Layout: arrays are indexed ``[y, x]`` (2D) or ``[z, y, x]`` (3D), x fastest.
Poisson grids are vertex-centred on the unit domain: node ``i`` (0-based) of
an ``N``-node axis sits at ``(i + 1) * h`` with ``h = 1 / (N + 1)``, so the
zero padding of the paper's filters lands on the boundary nodes.
"""
import numpy as np

__all__ = [
    "node_coords", "poisson_spacing", "blob_rhs", "manufactured_rhs",
    "random_solid_mask", "flood_fill_unreachable", "block_mask",
    "ns_initial_velocity", "batched_sides",
]


def poisson_spacing(shape):
    """Spacing per axis (x, y[, z]) of a vertex-centred unit-domain grid."""
    return tuple(1.0 / (n + 1) for n in reversed(shape))


def node_coords(shape):
    """Coordinates of the nodes, one array per geometric axis (x, y[, z]),
    each broadcast to ``shape``."""
    dim = len(shape)
    coords = []
    for a in range(dim):
        ax = dim - 1 - a
        n = shape[ax]
        c = (np.arange(n) + 1.0) / (n + 1)
        sh = [1] * dim
        sh[ax] = n
        coords.append(np.broadcast_to(c.reshape(sh), shape))
    return coords


def blob_rhs(shape, seed, n_blobs=8, solid=None, zero_mean=True):
    """Sum of ``n_blobs`` Gaussian blobs ``amp * exp(-|x - c|^2 / (2 w^2))``.

    Per blob the draws are, in this order: amp ~ U(-1, 1), w ~ U(0.02, 0.1),
    centre ~ U(0.1, 0.9)^dim (x first).  The field is zeroed on solid cells
    and, if ``zero_mean``, made zero-mean over the fluid cells in float64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dim = len(shape)
    f = np.zeros(shape)
    for _ in range(n_blobs):
        amp = rng.uniform(-1.0, 1.0)
        w = rng.uniform(0.02, 0.1)
        c = rng.uniform(0.1, 0.9, size=dim)
        # the Gaussian factorises over the axes: a product of 1D profiles
        g = np.full(shape, amp)
        for a in range(dim):
            ax = dim - 1 - a
            n = shape[ax]
            xa = (np.arange(n) + 1.0) / (n + 1)
            sh = [1] * dim
            sh[ax] = n
            g = g * np.exp(-((xa - c[a]) ** 2) / (2.0 * w * w)).reshape(sh)
        f = f + g
    fluid = np.ones(shape, bool) if solid is None else ~np.asarray(solid, bool)
    f = f * fluid
    if zero_mean and fluid.any():
        f = f - fluid * (f[fluid].mean())
    return f


def manufactured_rhs(shape):
    """dim * pi^2 * prod_a sin(pi x_a): the continuous -Laplacian of
    prod sin(pi x_a) on the unit domain, sampled at the nodes."""
    X = node_coords(shape)
    f = np.ones(shape)
    for c in X:
        f = f * np.sin(np.pi * c)
    return len(shape) * np.pi ** 2 * f


def flood_fill_unreachable(solid, bc):
    """Turn solid every fluid cell that cannot reach a Dirichlet face through
    face-adjacent fluid cells, so each fluid component touches a Dirichlet
    boundary and the pressure system stays nonsingular.  ``bc`` lists the
    face types x-, x+, y-, y+[, z-, z+] with 0 = Dirichlet."""
    solid = np.asarray(solid, bool).copy()
    fluid = ~solid
    dim = solid.ndim
    try:
        from scipy import ndimage
    except ImportError:
        ndimage = None
    if ndimage is not None:
        # face-connected fluid components; keep those touching a Dirichlet face
        lab, _ = ndimage.label(fluid)
        keep = set()
        for a in range(dim):
            ax = dim - 1 - a
            for side in (0, 1):
                if bc[2 * a + side] != 0:
                    continue
                sl = [slice(None)] * dim
                sl[ax] = 0 if side == 0 else -1
                keep.update(np.unique(lab[tuple(sl)]).tolist())
        keep.discard(0)
        reach = np.isin(lab, np.array(sorted(keep), dtype=lab.dtype)) & fluid
        return solid | (fluid & ~reach)
    reach = np.zeros_like(fluid)
    frontier = np.zeros_like(fluid)
    for a in range(dim):
        ax = dim - 1 - a
        for side in (0, 1):
            if bc[2 * a + side] != 0:
                continue
            sl = [slice(None)] * dim
            sl[ax] = 0 if side == 0 else -1
            frontier[tuple(sl)] |= fluid[tuple(sl)]
    reach |= frontier
    while frontier.any():
        grown = np.zeros_like(frontier)
        for ax in range(dim):
            n = solid.shape[ax]
            lo = [slice(None)] * dim
            hi = [slice(None)] * dim
            lo[ax] = slice(0, n - 1)
            hi[ax] = slice(1, n)
            grown[tuple(lo)] |= frontier[tuple(hi)]
            grown[tuple(hi)] |= frontier[tuple(lo)]
        frontier = grown & fluid & ~reach
        reach |= frontier
    return solid | (fluid & ~reach)


def random_solid_mask(shape, rng, frac, bc=(0, 0, 0, 0)):
    """Union of random axis-aligned rectangles (sides 2 .. N/8) added until
    the solid fraction reaches ``frac``; then flood-filled so every fluid
    cell reaches a Dirichlet face.  ``rng`` is a numpy Generator."""
    ny, nx = shape
    solid = np.zeros(shape, bool)
    target = frac * nx * ny
    smax_x, smax_y = max(2, nx // 8), max(2, ny // 8)
    while solid.sum() < target:
        wx = int(rng.integers(2, smax_x + 1))
        wy = int(rng.integers(2, smax_y + 1))
        x0 = int(rng.integers(0, nx - wx + 1))
        y0 = int(rng.integers(0, ny - wy + 1))
        solid[y0:y0 + wy, x0:x0 + wx] = True
    return flood_fill_unreachable(solid, bc)


def batched_sides(count, seed, choices=(64, 128, 256, 512)):
    """Side lengths of ``count`` square instances drawn uniformly from
    ``choices``, plus each instance's solid fraction ~ U(0, 0.10)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = rng.choice(np.asarray(choices), size=count)
    fracs = rng.uniform(0.0, 0.10, size=count)
    return [int(s) for s in sides], [float(f) for f in fracs], rng


def block_mask(cells, centre, side):
    """Solid cube/square of ``side`` cells centred on cell-corner ``centre``
    (x, y[, z]) in a grid of ``cells`` = (nx, ny[, nz]); returns an array
    indexed [y, x] / [z, y, x]."""
    dim = len(cells)
    shape = tuple(reversed(cells))
    solid = np.ones(shape, bool)
    for a in range(dim):
        ax = dim - 1 - a
        lo = int(centre[a]) - side // 2
        idx = np.arange(cells[a])
        m = (idx >= lo) & (idx < lo + side)
        sh = [1] * dim
        sh[ax] = cells[a]
        solid = solid & m.reshape(sh)
    return solid


def ns_initial_velocity(cells, seed, u_inflow=1.0, noise=0.01):
    """Staggered (MAC) initial velocity: u = u_inflow + noise * N(0, 1) on the
    x-faces, v (and w) = noise * N(0, 1) on their faces.  Draw order: u, v,
    w.  Shapes: u (.., ny, nx+1), v (.., ny+1, nx), w (nz+1, ny, nx)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dim = len(cells)
    if dim == 2:
        nx, ny = cells
        shapes = [(ny, nx + 1), (ny + 1, nx)]
    else:
        nx, ny, nz = cells
        shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    out = []
    for a, sh in enumerate(shapes):
        base = u_inflow if a == 0 else 0.0
        out.append(base + noise * rng.standard_normal(sh))
    return out


def convnet_weights(seed, layer_io=((2, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16),
                                    (16, 1)), last_scale=1.0):
    """He-normal initial weights of the 9 bias-free 3x3x3 convolutions of the
    initial-guess network: arrays [27, Cin, Cout] with std sqrt(2 / (27 Cin))
    (seeded; drawn layer by layer); the last layer is multiplied by
    last_scale (a small value starts training from a near-zero guess)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = [rng.standard_normal((27, ci, co)) * np.sqrt(2.0 / (27 * ci)) for ci, co in layer_io]
    w[-1] = w[-1] * last_scale
    return w


def advdiff_gaussian(shape, gamma=10.0, centre=(0.0, 0.0)):
    """The Gaussian initial condition of the advection-diffusion tests (Eq.
    Gaussian_distribution_T, its first term): exp(-((x - x0)^2 + (y -
    y0)^2) / (2 gamma^2)) on nodes x_l = l - (n - 1) / 2, y likewise (the
    domain centred on the origin, spacing 1), float64 array [y, x]."""
    ny, nx = shape
    x = np.arange(nx) - (nx - 1) / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    X, Y = np.meshgrid(x, y)
    return np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / (2.0 * gamma * gamma))
