"""FP64 oracle: one projection time step (Algorithm 1) on a staggered grid.

Test infrastructure only (see the package docstring).

Grid: ``cells = (nx, ny[, nz])`` cells of side ``h``.  Pressure sits at cell
centres (array ``[y, x]`` / ``[z, y, x]``).  Velocity component ``c`` sits on
the faces normal to axis ``c`` (a MAC arrangement): u has shape
``(.., ny, nx+1)``, v ``(.., ny+1, nx)``, w ``(nz+1, ny, nx)``; face ``f``
along ``c`` lies between cells ``f-1`` and ``f``.

Boundaries (flow past a bluff body): x- is an inflow (u = u_in, tangential
components 0), x+ an outflow (zero-gradient velocity, pressure 0), all other
faces free-slip walls (normal component 0, zero-gradient tangential
components, zero-gradient pressure).  Ghost values follow the paper's
padding rule (Sec. 2.3): a Dirichlet side pads with the specified value, a
zero-derivative side pads with the adjacent value.

Solid body: cells flagged solid.  Faces touching a solid cell carry the
absorption ``sigma`` treated implicitly (Eq. predictor-Burgers / Tn+1), which
drives them to 0; in the pressure equation solid cells are not unknowns and
fluid/solid faces are zero-gradient.

Step (Algorithm 1, with the readings used here):
1. momentum, predictor then corrector:
   ``(1 + sigma dt) q_new = q^n - dt [ sum_b U_b^n d_b Q + nu A_nu Q + d_c p^n ]``
   with ``Q = q^n`` (predictor) and ``Q = (q~ + q^n) / 2`` (corrector);
   ``U_b^n`` is the frozen advecting velocity at time n (Alg. 1, step 1),
   ``d_b`` the central difference (filters A^u, A^v of Eq. AAA), ``A_nu`` the
   5/7-point diffusion filter (App. A) divided by h^2; or, as an option, the
   finite-element 9/27-point filters of App. A (``momentum_rate_fe``);
2. pressure correction ``A_h dp = -(1/dt) D q*``, where the paper's
   "nabla^2" is its diffusion filter, i.e. ``A_h = -Laplacian_h`` (Sec. 2.1),
   and on the staggered grid ``A_h = -D G`` exactly;
3. ``q <- q* - dt G dp``;  4. ``p <- p + dp``.
"""
import itertools

import numpy as np

from . import poisson as P


def _take(f, ax, lo, hi):
    sl = [slice(None)] * f.ndim
    sl[ax] = slice(lo, hi)
    return f[tuple(sl)]


def pad(f, a, lo_mode, hi_mode):
    """Pad ``f`` by one layer on both sides of geometric axis ``a``;
    mode 'zero' = specified value 0, 'copy' = adjacent value."""
    ax = f.ndim - 1 - a
    n = f.shape[ax]
    lo = np.zeros_like(_take(f, ax, 0, 1)) if lo_mode == 'zero' else _take(f, ax, 0, 1)
    hi = np.zeros_like(_take(f, ax, n - 1, n)) if hi_mode == 'zero' else _take(f, ax, n - 1, n)
    return np.concatenate([lo, f, hi], axis=ax)


def ghost_modes(c, a):
    """Ghost rule of velocity component ``c`` along axis ``a``: the inflow
    side pads tangential components with 0; every other side copies."""
    lo = 'zero' if (a == 0 and c != 0) else 'copy'
    return lo, 'copy'


def shift(Qp, a, off):
    """From an array padded along axis ``a``, the values at offset ``off``
    (-1, 0, +1) for every interior index."""
    ax = Qp.ndim - 1 - a
    n = Qp.shape[ax] - 2
    return _take(Qp, ax, 1 + off, 1 + off + n)


class MacGrid:
    """Geometry, masks and the three operators D, G, A of the projection."""

    def __init__(self, cells, h, solid, sigma=1e8):
        self.cells = tuple(int(v) for v in cells)
        self.dim = len(self.cells)
        self.h = float(h)
        self.shape = tuple(reversed(self.cells))
        self.solid = np.zeros(self.shape, bool) if solid is None else np.asarray(solid, bool)
        self.sigma = float(sigma)
        # pressure BCs: x- Neumann, x+ Dirichlet (p = 0), walls Neumann
        self.p_bc = tuple([1, 0] + [1, 1] * (self.dim - 1))
        self.level = P.Level(self.shape, (self.h,) * self.dim, self.p_bc, self.solid)

    def face_shape(self, c):
        s = list(self.shape)
        s[self.dim - 1 - c] += 1
        return tuple(s)

    def face_index(self, c):
        """Index of every c-face along axis c, broadcast to the face array."""
        ax = self.dim - 1 - c
        n = self.cells[c] + 1
        sh = [1] * self.dim
        sh[ax] = n
        return np.broadcast_to(np.arange(n).reshape(sh), self.face_shape(c))

    def fixed_faces(self, c):
        """Faces whose value is prescribed: the inflow face of u; both wall
        faces of v and w."""
        f = self.face_index(c)
        if c == 0:
            return f == 0
        return (f == 0) | (f == self.cells[c])

    def solid_face(self, c):
        """Faces that touch a solid cell (either side)."""
        sp = pad(self.solid, c, 'copy', 'copy')
        return self._face_pair_any(sp, c)

    def _face_pair_any(self, sp, c):
        ax = self.dim - 1 - c
        n = self.cells[c] + 1
        left = _take(sp, ax, 0, n)        # cell f-1
        right = _take(sp, ax, 1, n + 1)   # cell f
        return left | right

    def correctable(self, c):
        """Faces that the pressure gradient corrects: interior faces between
        two fluid cells, and the outflow faces of u next to a fluid cell."""
        fluid = ~self.solid
        ax = self.dim - 1 - c
        n = self.cells[c] + 1
        fp = pad(fluid, c, 'zero', 'copy' if c == 0 else 'zero')
        left = _take(fp, ax, 0, n)
        right = _take(fp, ax, 1, n + 1)
        ok = left & right
        f = self.face_index(c)
        ok = ok & (f > 0)
        if c != 0:
            ok = ok & (f < self.cells[c])
        return ok

    # -- operators ---------------------------------------------------------
    def divergence(self, q):
        """D q at every cell: sum_c (q_c[f+1] - q_c[f]) / h."""
        d = np.zeros(self.shape)
        for c in range(self.dim):
            ax = self.dim - 1 - c
            n = self.cells[c]
            d = d + (_take(q[c], ax, 1, n + 1) - _take(q[c], ax, 0, n)) / self.h
        return d

    def gradient(self, dp):
        """G dp on the correctable faces, 0 elsewhere; the outflow ghost of
        the pressure is 0 (Dirichlet)."""
        out = []
        for c in range(self.dim):
            ax = self.dim - 1 - c
            n = self.cells[c] + 1
            pp = pad(dp, c, 'copy', 'zero' if c == 0 else 'copy')
            g = (_take(pp, ax, 1, n + 1) - _take(pp, ax, 0, n)) / self.h
            out.append(np.where(self.correctable(c), g, 0.0))
        return out

    def pressure_gradient(self, p):
        """d_c p at every face (momentum source -grad p^n); the outflow ghost
        is 0, the other ghosts copy (zero gradient)."""
        out = []
        for c in range(self.dim):
            ax = self.dim - 1 - c
            n = self.cells[c] + 1
            pp = pad(p, c, 'copy', 'zero' if c == 0 else 'copy')
            out.append((_take(pp, ax, 1, n + 1) - _take(pp, ax, 0, n)) / self.h)
        return out


def advecting_velocity(g, q, c, b):
    """Component ``b`` of the time-n velocity at the faces of component
    ``c``: q_c itself if b == c, else the average of the four q_b values
    around the c-face (two cells along c, two faces along b)."""
    if b == c:
        return q[c]
    lo, hi = ghost_modes(b, c)
    qp = pad(q[b], c, lo, hi)
    axc = g.dim - 1 - c
    axb = g.dim - 1 - b
    nc = g.cells[c] + 1
    nb = g.cells[b]
    s = _take(qp, axc, 0, nc) + _take(qp, axc, 1, nc + 1)     # cells f-1, f
    s = _take(s, axb, 0, nb) + _take(s, axb, 1, nb + 1)        # faces j, j+1
    return 0.25 * s


def momentum_rate(g, q, c, Q, U, nu, gradp):
    """Bracket of Eq. predictor-Burgers for component c evaluated on Q:
    sum_b U_b d_b Q + nu A_nu Q + d_c p^n."""
    h = g.h
    adv = np.zeros_like(Q)
    diff = np.zeros_like(Q)
    for a in range(g.dim):
        lo, hi = ghost_modes(c, a)
        Qp = pad(Q, a, lo, hi)
        qm, q0, qpl = shift(Qp, a, -1), shift(Qp, a, 0), shift(Qp, a, +1)
        adv = adv + U[a] * (qpl - qm) / (2.0 * h)
        diff = diff + (2.0 * q0 - qm - qpl) / (h * h)
    return adv + nu * diff + gradp[c]


def _pad_all(g, c, Q):
    """Q padded by one layer along every axis, each axis by component c's
    ghost rule in turn (so a corner ghost follows both rules)."""
    Qp = Q
    for a in range(g.dim):
        lo, hi = ghost_modes(c, a)
        Qp = pad(Qp, a, lo, hi)
    return Qp


def _at(Qp, off):
    """From an array padded along every axis, the values at offset ``off``
    = (ox, oy[, oz]) for every interior index."""
    sl = []
    for ax in range(Qp.ndim):
        a = Qp.ndim - 1 - ax
        n = Qp.shape[ax] - 2
        sl.append(slice(1 + off[a], 1 + off[a] + n))
    return Qp[tuple(sl)]


def fe_diffusion_weights(dim):
    """The paper's finite-element diffusion filters (App. A) as
    {offset: weight} with their common factor: 2D 9-point 1/(4 h^2) x
    [-1 -2 -1; -2 12 -2; -1 -2 -1]; 3D 27-point 1/(26 h^2) x (centre 88,
    -6 on the 6 face neighbours, -3 on the 12 edge neighbours, -2 on the 8
    corners).  The weight depends on how many offset components are
    non-zero."""
    by_count = {2: {0: 12.0, 1: -2.0, 2: -1.0}, 3: {0: 88.0, 1: -6.0, 2: -3.0, 3: -2.0}}[dim]
    scale = {2: 4.0, 3: 26.0}[dim]
    w = {}
    for off in itertools.product((-1, 0, 1), repeat=dim):
        w[off] = by_count[sum(1 for o in off if o != 0)]
    return w, scale


def fe_advection_weights(dim, a):
    """The paper's finite-element advection filters along axis ``a`` (App.
    A) as {offset: weight} and their factor: the central difference along
    ``a`` smoothed by (1, 4, 1) across each other axis; 2D 1/(12 h), 3D
    1/(72 h).  The sign is + towards +a on every axis (the printed z filter
    of the paper carries the opposite sign; read as the same filter)."""
    side = {-1: 1.0, 0: 4.0, 1: 1.0}
    w = {}
    for off in itertools.product((-1, 0, 1), repeat=dim):
        if off[a] == 0:
            continue
        v = float(off[a])
        for b in range(dim):
            if b != a:
                v *= side[off[b]]
        w[off] = v
    return w, {2: 12.0, 3: 72.0}[dim]


def momentum_rate_fe(g, q, c, Q, U, nu, gradp):
    """Bracket of Eq. predictor-Burgers with the paper's finite-element
    filters (App. A: 9-point / 27-point diffusion, the advection filters),
    applied to component c on its own face grid: sum_b U_b d_b^FE Q +
    nu A_nu^FE Q + d_c p^n."""
    h = g.h
    Qp = _pad_all(g, c, Q)
    wd, sd = fe_diffusion_weights(g.dim)
    diff = np.zeros_like(Q)
    for off, w in wd.items():
        diff = diff + w * _at(Qp, off)
    diff = diff / (sd * h * h)
    adv = np.zeros_like(Q)
    for a in range(g.dim):
        wa, sa = fe_advection_weights(g.dim, a)
        da = np.zeros_like(Q)
        for off, w in wa.items():
            da = da + w * _at(Qp, off)
        adv = adv + U[a] * da / (sa * h)
    return adv + nu * diff + gradp[c]


def momentum(g, q, p, dt, nu, u_inflow, fe=False):
    """Step 1 of Algorithm 1: predictor, then corrector.  Returns q*.
    ``fe`` selects the finite-element filters (``momentum_rate_fe``)."""
    rate_fn = momentum_rate_fe if fe else momentum_rate
    q = enforce_bc(g, q, u_inflow)
    gradp = g.pressure_gradient(p)
    U = {c: [advecting_velocity(g, q, c, b) for b in range(g.dim)] for c in range(g.dim)}
    denom = [1.0 + np.where(g.solid_face(c), g.sigma, 0.0) * dt for c in range(g.dim)]
    fixed = [g.fixed_faces(c) for c in range(g.dim)]
    pred = []
    for c in range(g.dim):
        rate = rate_fn(g, q, c, q[c], U[c], nu, gradp)
        new = (q[c] - dt * rate) / denom[c]
        pred.append(np.where(fixed[c], q[c], new))
    out = []
    for c in range(g.dim):
        Q = 0.5 * (pred[c] + q[c])
        rate = rate_fn(g, q, c, Q, U[c], nu, gradp)
        new = (q[c] - dt * rate) / denom[c]
        out.append(np.where(fixed[c], q[c], new))
    return out


def enforce_bc(g, q, u_inflow):
    """Set the prescribed faces: u = u_in on the inflow, v = w = 0 on the
    walls."""
    out = [np.array(a, dtype=np.float64, copy=True) for a in q]
    for c in range(g.dim):
        fx = g.fixed_faces(c)
        out[c][fx] = u_inflow if c == 0 else 0.0
    return out


def divergence_rhs(g, qs, dt):
    """Step 2 right-hand side: b = -(1/dt) D q* on fluid cells."""
    return -(1.0 / dt) * g.divergence(qs) * (~g.solid)


def correct(g, qs, p, dp, dt):
    """Steps 3-5: q = q* - dt G dp, p = p + dp."""
    G = g.gradient(dp)
    return [qs[c] - dt * G[c] for c in range(g.dim)], p + dp


def ns_step(g, q, p, dt, nu, u_inflow, tol=1e-12, solve=None, fe=False):
    """One full step of Algorithm 1.  The pressure correction is solved to
    relative residual ``tol`` (default 1e-12) by ``solve(b)`` if given, else
    by the oracle's dense solve (small grids) or MG-PCG.  ``fe`` selects the
    finite-element momentum filters of App. A.
    Returns (q_new, p_new, dp, q_star, b)."""
    qs = momentum(g, q, p, dt, nu, u_inflow, fe=fe)
    b = divergence_rhs(g, qs, dt)
    if solve is None:
        dp = P.solve_reference(g.shape, (g.h,) * g.dim, g.p_bc, b, g.solid, tol=tol, s=1.0)
    else:
        dp = solve(b)
    qn, pn = correct(g, qs, p, dp, dt)
    return qn, pn, dp, qs, b
