"""FP64 oracle: one implicit backward-Euler step of the advection-diffusion
equation (Eq. adv-diff-eqn with s = sigma = 0; Eq. BE-advection-concise)
and its multigrid solution (Sec. 2.2 cycle, Sec. 3.2 "Multigrid solver for
the advection-diffusion equation").

Test infrastructure only (see the package docstring).

Field layout: a 2D array ``[y, x]`` (x fastest) of nodes with spacing ``h``;
zero padding on every side (Sec. 2.1: a zero solution on the boundary).

One step solves ``A T^{n+1} = T^n`` with

    A T = T + dt ( u d_x T + v d_y T - nu Lap_h T )

for constant (u, v) and nu: the identity filter plus dt times the advection
filters (central: Eq. A; upwind: Eq. A-up) plus dt times the 5-point
diffusion filter (App. A), applied as a cross-correlation (Eq.
define_convolution).  ``d_x`` is the central difference (T_{l+1} -
T_{l-1}) / 2h, or the first-order upwind difference: backward (T_l -
T_{l-1}) / h for u >= 0, forward for u < 0.  The printed upwind filter
(Eq. A-up) holds the forward differences; it is the upwind one for a
velocity along -x and -y, and for (u, v) = (1, 1) this module takes its
mirror image, the backward differences (the upwind scheme for that
velocity; the test files pin both facts).

Every level holds a constant 5-point stencil ``(c, xm, xp, ym, yp)``:
``(A T)_l = c T_l + xm T_{l-1} + xp T_{l+1} + ym T_{m-1} + yp T_{m+1}``.
Coarse levels (spacing 2^k h) either re-discretise the operator
(``coarse='rediscretise'``, App. B: the filters change with the spacing) or
take the Galerkin product R A P of the average restriction and copy
prolongation, which for these filters is the re-discretised stencil with
the diffusion term multiplied by 2^k (``coarse='galerkin'``; pinned against
the dense product).
"""
import numpy as np

from .poisson import neighbour, restrict


def stencil(h, dt, nu, u, v, scheme, diff_scale=1.0):
    """Weights (c, xm, xp, ym, yp) of A at spacing h; ``diff_scale``
    multiplies the diffusion term (1 = the re-discretised filter)."""
    kd = diff_scale * nu * dt / (h * h)
    c, xm, xp, ym, yp = 1.0 + 4.0 * kd, -kd, -kd, -kd, -kd
    if scheme == 'central':
        ax, ay = u * dt / (2.0 * h), v * dt / (2.0 * h)
        xm, xp, ym, yp = xm - ax, xp + ax, ym - ay, yp + ay
    elif scheme == 'upwind':
        cx, cy = u * dt / h, v * dt / h
        if u >= 0:
            c, xm = c + cx, xm - cx
        else:
            c, xp = c - cx, xp + cx
        if v >= 0:
            c, ym = c + cy, ym - cy
        else:
            c, yp = c - cy, yp + cy
    else:
        raise ValueError(scheme)
    return (c, xm, xp, ym, yp)


class ADLevel:
    """One grid of the hierarchy: its shape and constant stencil."""

    def __init__(self, shape, w):
        self.shape = tuple(int(s) for s in shape)
        self.w = tuple(float(t) for t in w)

    def apply(self, x):
        """A x with zero padding (Eq. define_convolution)."""
        c, xm, xp, ym, yp = self.w
        return (c * x + xm * neighbour(x, 0, -1) + xp * neighbour(x, 0, +1)
                + ym * neighbour(x, 1, -1) + yp * neighbour(x, 1, +1))

    def dense(self):
        """Dense matrix of A (C order over [y, x]), built node by node from
        the stencil with the zero-padding rule."""
        ny, nx = self.shape
        c, xm, xp, ym, yp = self.w
        A = np.zeros((nx * ny, nx * ny))
        for j in range(ny):
            for i in range(nx):
                r = j * nx + i
                A[r, r] = c
                for di, dj, wt in ((-1, 0, xm), (1, 0, xp), (0, -1, ym), (0, 1, yp)):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < nx and 0 <= jj < ny:
                        A[r, jj * nx + ii] += wt
        return A


def build_hierarchy(shape, h, dt, nu, u, v, scheme='upwind', coarse='rediscretise', levels=0, coarsest_max=4):
    """Level 0 = finest; spacing 2^k h on level k.  ``levels=0`` coarsens
    while both sides stay even and the halved side is >= ``coarsest_max``."""
    shape = tuple(int(s) for s in shape)
    if levels <= 0:
        levels = 1
        s = shape
        while all(t % 2 == 0 and t // 2 >= coarsest_max for t in s):
            s = tuple(t // 2 for t in s)
            levels += 1
    hier = []
    for k in range(levels):
        assert all(t % (1 << k) == 0 for t in shape)
        scale = float(1 << k) if coarse == 'galerkin' else 1.0
        hier.append(ADLevel(tuple(t >> k for t in shape), stencil(h * (1 << k), dt, nu, u, v, scheme, scale)))
    return hier


def prolong(e):
    """Copy each coarse value to its 2x2 children (Sec. 2.2)."""
    return np.repeat(np.repeat(e, 2, axis=0), 2, axis=1)


def jacobi(lv, x, b, omega):
    """One relaxed Jacobi sweep (Eq. Jacobi-1-relax): x + omega (b - A x) / c."""
    return x + omega * (b - lv.apply(x)) / lv.w[0]


def residual(lv, b, x):
    return b - lv.apply(x)


def relres(lv, b, x):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(residual(lv, b, x)) / (nb if nb > 0 else 1.0))


def dense_solve(lv, b):
    """The definition of one step's answer: T^{n+1} = A^{-1} T^n (numpy LU)."""
    return np.linalg.solve(lv.dense(), b.ravel()).reshape(lv.shape)


class ADMultigrid:
    """The cycles of Sec. 2.2 / App. B on an advection-diffusion hierarchy.

    ``'V'``: ``pre`` relaxed Jacobi sweeps from zero, the residual averaged
    to the next level, recursion from zero, ``s`` times the copied
    correction added, ``post`` sweeps; the coarsest level solved densely.
    ``'sawtooth'``: the residual restricted without smoothing; from the
    coarsest level up, r/c plus ``s`` times the copied correction of the
    level below, then ``post`` relaxed Jacobi sweeps (the paper's cycle,
    with its alpha = 1 and one sweep as ``omega = 1, post = 1``)."""

    def __init__(self, hier, cycle='sawtooth', pre=1, post=1, omega=1.0, s=1.0):
        self.hier, self.cycle = hier, cycle
        self.pre, self.post, self.omega, self.s = pre, post, omega, s
        self.coarse_A = hier[-1].dense()

    def v_level(self, k, b):
        lv = self.hier[k]
        if k == len(self.hier) - 1:
            return np.linalg.solve(self.coarse_A, b.ravel()).reshape(lv.shape)
        x = np.zeros_like(b)
        for _ in range(self.pre):
            x = jacobi(lv, x, b, self.omega)
        e = self.v_level(k + 1, restrict(residual(lv, b, x)))
        x = x + self.s * prolong(e)
        for _ in range(self.post):
            x = jacobi(lv, x, b, self.omega)
        return x

    def saw_level(self, k, r):
        lv = self.hier[k]
        x = r / lv.w[0]
        if k < len(self.hier) - 1:
            x = x + self.s * prolong(self.saw_level(k + 1, restrict(r)))
        for _ in range(self.post):
            x = jacobi(lv, x, r, self.omega)
        return x

    def precondition(self, r):
        """z = M r: one cycle from a zero guess."""
        return self.saw_level(0, r) if self.cycle == 'sawtooth' else self.v_level(0, r)

    def solve(self, b, x0=None, tol=1e-6, l1_tol=0.0, max_cycles=1000):
        """Stationary iteration x <- x + M (b - A x) from ``x0`` (default
        b, i.e. T^n: the previous time level, Sec. 3.2).  Stops when
        ||b - A x||_2 / ||b||_2 <= tol, or when the L1 norm of the change of
        x over one cycle is <= l1_tol (the paper's gauge, Sec. 3.2), or
        after max_cycles.  Returns (x, cycles, relres history, L1 history)."""
        lv = self.hier[0]
        x = (b.copy() if x0 is None else x0.copy()).astype(np.float64)
        rr, l1 = [relres(lv, b, x)], []
        k = 0
        while k < max_cycles and rr[-1] > tol:
            z = self.precondition(residual(lv, b, x))
            x = x + z
            k += 1
            rr.append(relres(lv, b, x))
            l1.append(float(np.abs(z).sum()))
            if l1[-1] <= l1_tol:
                break
        return x, k, rr, l1

