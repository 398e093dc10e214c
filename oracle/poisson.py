"""FP64 oracle: discrete pressure-Poisson operator and its multigrid solver.

Test infrastructure only (see the package docstring): the GPU library never
uses this module.

Conventions (shared with the GPU library's public header, not its code):

* A field is a numpy array indexed ``[y, x]`` (2D) or ``[z, y, x]`` (3D),
  x fastest.  Axis number ``a`` (0 = x, 1 = y, 2 = z) is array axis
  ``ndim - 1 - a``.
* ``h`` is the spacing per axis ``(hx, hy[, hz])``.
* ``bc`` lists ``2 * dim`` face types in the order x-, x+, y-, y+, z-, z+;
  0 = Dirichlet (ghost value 0, the paper's zero padding of Sec. 2.1),
  1 = homogeneous Neumann (ghost = copy of the adjacent value, Sec. 2.3).
* ``solid`` is a bool array (True = solid cell) or None.  Solid cells are not
  unknowns: they hold 0 and a fluid/solid face is treated as homogeneous
  Neumann (the link is dropped and the diagonal reduced).
* The operator is the paper's diffusion filter with unit coefficient,
  ``A_h = -Laplacian_h`` (App. A: 2D 5-point [0 -1 0; -1 4 -1; 0 -1 0]/h^2,
  3D 7-point with centre 6), applied as a cross-correlation (Eq.
  define_convolution).  With Dirichlet ghosts at 0 it is SPD.
"""
import numpy as np


# --------------------------------------------------------------------------
# Geometry helpers
# --------------------------------------------------------------------------

def array_axis(ndim, a):
    """Array axis that carries geometric axis ``a`` (0 = x fastest)."""
    return ndim - 1 - a


def neighbour(f, a, off):
    """Value of ``f`` at the neighbour ``off`` (+1/-1) along geometric axis
    ``a``, with 0 outside the array -- the zero padding of Sec. 2.1."""
    ax = array_axis(f.ndim, a)
    n = f.shape[ax]
    out = np.zeros_like(f)
    dst = [slice(None)] * f.ndim
    src = [slice(None)] * f.ndim
    if off > 0:
        dst[ax] = slice(0, n - 1)
        src[ax] = slice(1, n)
    else:
        dst[ax] = slice(1, n)
        src[ax] = slice(0, n - 1)
    out[tuple(dst)] = f[tuple(src)]
    return out


class Level:
    """One grid of the hierarchy: fluid flags, off-diagonal links and the
    diagonal of A_h (Sec. 2.1 filters; Sec. 2.3 padding rules for BCs).

    ``link[(a, off)]`` is 1 where the cell and its neighbour along axis ``a``
    (direction ``off``) are both fluid cells inside the domain: those pairs
    couple with weight -1/h_a^2.  The diagonal counts, per axis, the coupled
    neighbours plus the domain faces whose BC is Dirichlet, times 1/h_a^2.
    """

    def __init__(self, shape, h, bc, solid=None):
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        self.h = tuple(float(v) for v in h)
        self.bc = tuple(int(v) for v in bc)
        assert len(self.h) == self.dim and len(self.bc) == 2 * self.dim
        if solid is None:
            solid = np.zeros(self.shape, dtype=bool)
        self.solid = np.asarray(solid, dtype=bool)
        self.fluid = (~self.solid).astype(np.float64)
        ones = np.ones(self.shape)
        self.link = {}
        diag = np.zeros(self.shape)
        for a in range(self.dim):
            inv_h2 = 1.0 / self.h[a] ** 2
            for side, off in ((0, -1), (1, +1)):
                inside = neighbour(ones, a, off)            # neighbour exists
                nb_fluid = neighbour(self.fluid, a, off)    # 0 outside
                lk = self.fluid * nb_fluid
                dirichlet_face = self.fluid * (1.0 - inside) * (self.bc[2 * a + side] == 0)
                self.link[(a, off)] = lk
                diag += (lk + dirichlet_face) * inv_h2
        self.diag = diag

    @property
    def n_unknowns(self):
        return int(self.fluid.sum())


def apply_A(lv, x):
    """(A_h x) on every fluid cell, 0 on solid cells (Sec. 2.1, App. A)."""
    y = lv.diag * x
    for a in range(lv.dim):
        inv_h2 = 1.0 / lv.h[a] ** 2
        for off in (-1, +1):
            y = y - lv.link[(a, off)] * neighbour(x, a, off) * inv_h2
    return y * lv.fluid


def residual(lv, b, x):
    """r = b - A_h x on fluid cells (App. B, the residual on level 1)."""
    return (b - apply_A(lv, x)) * lv.fluid


def relres(lv, b, x):
    """||b - A x||_2 / ||b||_2 in float64."""
    nb = np.linalg.norm(b * lv.fluid)
    return float(np.linalg.norm(residual(lv, b, x)) / (nb if nb > 0 else 1.0))


# --------------------------------------------------------------------------
# Dense assembly (plain loops) -- the definition of the answer on small grids
# --------------------------------------------------------------------------

def fluid_index(lv):
    """Map cell multi-index -> row number over fluid cells (C order)."""
    idx = -np.ones(lv.shape, dtype=np.int64)
    flat = np.flatnonzero(~lv.solid.ravel())
    idx.ravel()[flat] = np.arange(flat.size)
    return idx


def assemble_dense(lv):
    """Dense matrix of A_h over the fluid cells, built cell by cell with
    Python loops straight from the stencil definition and the BC rules.  It
    does not reuse ``Level``'s arrays, so it cross-checks them."""
    idx = fluid_index(lv)
    n = int((idx >= 0).sum())
    A = np.zeros((n, n))
    for cell in np.ndindex(*lv.shape):
        row = idx[cell]
        if row < 0:
            continue
        for a in range(lv.dim):
            ax = array_axis(lv.dim, a)
            inv_h2 = 1.0 / lv.h[a] ** 2
            for side, off in ((0, -1), (1, +1)):
                nb = list(cell)
                nb[ax] += off
                if nb[ax] < 0 or nb[ax] >= lv.shape[ax]:
                    if lv.bc[2 * a + side] == 0:      # Dirichlet: ghost 0
                        A[row, row] += inv_h2
                    continue                          # Neumann: no link
                col = idx[tuple(nb)]
                if col < 0:                           # solid neighbour: Neumann
                    continue
                A[row, row] += inv_h2
                A[row, col] -= inv_h2
    return A


def dense_solve(lv, b, A=None):
    """x* = A_h^{-1} b on the fluid cells by a dense LU (numpy.linalg.solve),
    0 on solid cells.  This is the plain definition of the solve's result."""
    if A is None:
        A = assemble_dense(lv)
    mask = ~lv.solid.ravel()
    x = np.zeros(lv.shape)
    if A.shape[0]:
        x.ravel()[mask] = np.linalg.solve(A, b.ravel()[mask])
    return x


# --------------------------------------------------------------------------
# Multigrid building blocks (Sec. 2.2; App. B)
# --------------------------------------------------------------------------

def jacobi(lv, x, b, omega):
    """One relaxed Jacobi sweep, Eq. Jacobi-1-relax:
    x <- x + omega * D^{-1} (b - A x) on fluid cells."""
    d = np.where(lv.diag > 0, lv.diag, 1.0)
    return (x + omega * (b - apply_A(lv, x)) / d) * lv.fluid


def _blocks(f):
    """View ``f`` as coarse cells x 2^dim children (the 2x2(x2) filter of
    stride 2 in Sec. 2.2; children of coarse cell (l, m) are (2l..2l+1,
    2m..2m+1))."""
    if f.ndim == 2:
        ny, nx = f.shape
        return f.reshape(ny // 2, 2, nx // 2, 2), (1, 3)
    nz, ny, nx = f.shape
    return f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2), (1, 3, 5)


def restrict(r):
    """Average of the 2^dim children (Sec. 2.2: 2x2 filter of 1/4, stride 2;
    App. B: four quarters in 2D, eight eighths in 3D)."""
    v, axes = _blocks(r)
    return v.mean(axis=axes)


def prolong(e, fine_lv):
    """Copy each coarse value to its 2^dim children (Sec. 2.2: 2x2 filter of
    ones, stride 2); solid fine cells get 0."""
    out = e
    for ax in range(e.ndim):
        out = np.repeat(out, 2, axis=ax)
    return out * fine_lv.fluid


def coarsen_solid(solid):
    """A coarse cell is solid iff all its children are solid."""
    v, axes = _blocks(solid.astype(bool))
    return v.all(axis=axes)


def build_hierarchy(shape, h, bc, solid=None, levels=0, coarsest_max=4):
    """Level 0 = finest.  The spacing doubles per level (App. B: "the grid
    spacing changes between the layers", the coarse filters are the same
    stencils re-discretised at spacing 2^k h).  ``levels=0`` coarsens until
    the smallest side reaches ``coarsest_max``."""
    shape = tuple(int(s) for s in shape)
    if levels <= 0:
        levels = 1
        s = min(shape)
        while s % 2 == 0 and s // 2 >= coarsest_max:
            s //= 2
            levels += 1
    for s in shape:
        assert s % (1 << (levels - 1)) == 0, "side not divisible by 2^(levels-1)"
    hier = [Level(shape, h, bc, solid)]
    for _ in range(1, levels):
        prev = hier[-1]
        cshape = tuple(s // 2 for s in prev.shape)
        hier.append(Level(cshape, tuple(2 * v for v in prev.h), bc,
                          coarsen_solid(prev.solid)))
    return hier


class Multigrid:
    """Multigrid preconditioner / solver on a hierarchy (Sec. 2.2 step list).

    Cycle ``'V'``: on each level smooth ``pre`` times, restrict the residual,
    recurse from a zero guess, add ``s`` times the prolonged correction,
    smooth ``post`` times; the coarsest level is solved exactly by a dense LU.
    ``'W'`` recurses twice.  ``'sawtooth'`` is the paper's own cycle
    (``sawtooth_level``).  ``s`` is the coarse-correction scale (1 = the
    plain re-discretised correction).
    """

    def __init__(self, hier, pre=2, post=2, omega=2.0 / 3.0, s=0.7, cycle='V'):
        self.hier = hier
        self.pre, self.post, self.omega, self.s, self.cycle = pre, post, omega, s, cycle
        self.coarse_A = assemble_dense(hier[-1])

    def cycle_level(self, k, b, x):
        lv = self.hier[k]
        if k == len(self.hier) - 1:
            return dense_solve(lv, b, self.coarse_A)
        for _ in range(self.pre):
            x = jacobi(lv, x, b, self.omega)
        r = residual(lv, b, x)
        bc = restrict(r)
        nrec = 2 if (self.cycle == 'W' and k + 1 < len(self.hier) - 1) else 1
        ec = np.zeros_like(bc)
        for _ in range(nrec):
            ec = self.cycle_level(k + 1, bc, ec)
        x = x + self.s * prolong(ec, lv)
        for _ in range(self.post):
            x = jacobi(lv, x, b, self.omega)
        return x

    def sawtooth_level(self, k, r):
        """The paper's sawtooth cycle (App. B recursion, under the reading that
        Eq. e22 is a Jacobi step (r - A T) / A0): the level's residual is
        restricted to the next level without any smoothing (Eq. r-recur);
        then, from the coarsest level up, the level's correction is one
        Jacobi step from zero, r^k / d (Eq. e19), plus s times the prolonged
        correction of the level below (Eq. e20; at the coarsest level the
        Jacobi step alone, Eq. e20b), followed by ``post`` relaxed Jacobi
        sweeps on A x = r^k (Eqs. e21-e23).  No exact coarsest solve."""
        lv = self.hier[k]
        d = np.where(lv.diag > 0, lv.diag, 1.0)
        x = (r / d) * lv.fluid
        if k < len(self.hier) - 1:
            ec = self.sawtooth_level(k + 1, restrict(r))
            x = x + self.s * prolong(ec, lv)
        for _ in range(self.post):
            x = jacobi(lv, x, r, self.omega)
        return x

    def precondition(self, r):
        """z = M r: one cycle from a zero guess."""
        if self.cycle == 'sawtooth':
            return self.sawtooth_level(0, r)
        return self.cycle_level(0, r, np.zeros_like(r))

    def stationary(self, b, cycles, x0=None):
        """x <- x + M (b - A x), ``cycles`` times (the cycle as a solver);
        returns x and the relres after each cycle."""
        lv = self.hier[0]
        x = np.zeros_like(b) if x0 is None else x0.copy()
        hist = []
        for _ in range(cycles):
            x = x + self.precondition(residual(lv, b, x))
            hist.append(relres(lv, b, x))
        return x, hist


# --------------------------------------------------------------------------
# Krylov wrapper and iterative refinement
# --------------------------------------------------------------------------

def pcg(mg, b, x0=None, tol=1e-6, max_iters=500, rnorm_ref=None):
    """Preconditioned conjugate gradients on A_h with M = one symmetric
    multigrid cycle.  Stops when ||r||_2 <= tol * ||b||_2 (or ``rnorm_ref``).
    Returns (x, history of ||r||/ref, iterations).  The residual is updated
    by the recurrence r <- r - alpha A p, as in textbook CG."""
    lv = mg.hier[0]
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = residual(lv, b, x)
    ref = np.linalg.norm(b * lv.fluid) if rnorm_ref is None else rnorm_ref
    if ref == 0:
        return x, [0.0], 0
    hist = [np.linalg.norm(r) / ref]
    if hist[-1] <= tol:
        return x, hist, 0
    z = mg.precondition(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    it = 0
    while it < max_iters:
        Ap = apply_A(lv, p)
        alpha = rz / float(np.vdot(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        hist.append(np.linalg.norm(r) / ref)
        if hist[-1] <= tol:
            break
        z = mg.precondition(r)
        rz_new = float(np.vdot(r, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, hist, it


def inner_tolerance(tol, relres_outer, floor):
    """Relative tolerance of one inner solve of the refinement loop: just
    enough to reach ``tol`` (with a factor 2 margin), but no tighter than the
    inner precision's ``floor``."""
    return max(0.5 * tol / relres_outer, floor)


def pcg_ir(mg, b, x0=None, tol=1e-6, inner_floor=1e-4, max_outer=20,
           max_inner=500):
    """Iterative refinement around MG-PCG (the solve the GPU runs):
    x += PCG(A, b - A x) until ||b - A x|| <= tol ||b||.  Each inner solve
    starts from 0 and stops at relative tolerance ``inner_tolerance``.
    Returns (x, outer relres history, total inner iterations)."""
    lv = mg.hier[0]
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = np.linalg.norm(b * lv.fluid)
    hist, inner = [], 0
    for _ in range(max_outer + 1):
        r = residual(lv, b, x)
        rr = np.linalg.norm(r) / (nb if nb > 0 else 1.0)
        hist.append(rr)
        if rr <= tol or nb == 0:
            break
        eta = inner_tolerance(tol, rr, inner_floor)
        d, _, it = pcg(mg, r, tol=eta, max_iters=max_inner)
        inner += it
        x = x + d
    return x, hist, inner


def solve_reference(shape, h, bc, b, solid=None, tol=1e-12, s=0.7):
    """x* = A_h^{-1} b: dense LU when there are at most 4096 fluid cells,
    otherwise MG-PCG to relative residual ``tol`` (default 1e-12)."""
    lv = Level(shape, h, bc, solid)
    if lv.n_unknowns <= 4096:
        return dense_solve(lv, b)
    mg = Multigrid(build_hierarchy(shape, h, bc, solid), s=s)
    x, _, _ = pcg(mg, b * lv.fluid, tol=tol, max_iters=2000)
    return x
