"""Pins of the oracle's finite-element momentum filters (App. A: 9-point /
27-point diffusion, the smoothed central-difference advection filters)
against the printed filters, closed forms on polynomials and the reduction
to the 5/7-point filters on fields that vary along one axis (no GPU)."""
import itertools
import os

import numpy as np
import pytest

from oracle import ns as N
from paper_2402_17913_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fe_filters_appA.txt")


def _golden():
    out, name = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                name = line[1:line.index("]")]
                den = float(line.split("den=")[1])
                out[name] = [den, []]
            else:
                out[name][1].append([float(v) for v in line.split()])
    return {k: (d, np.array(rows)) for k, (d, rows) in out.items()}


def _as_array(wdict, dim):
    """Oracle weights as the printed layout: 2D [x][y]; 3D [slice z][x][y]."""
    if dim == 2:
        m = np.zeros((3, 3))
        for (ox, oy), w in wdict.items():
            m[ox + 1, oy + 1] = w
    else:
        m = np.zeros((3, 3, 3))
        for (ox, oy, oz), w in wdict.items():
            m[oz + 1, ox + 1, oy + 1] = w
    return m


@pytest.mark.parametrize("dim", [2, 3])
def test_filters_match_the_printed_filters(dim):
    """The diffusion and x/y advection filters equal App. A's printed
    matrices (rows along x, columns along y, slices along z) with their
    printed denominators; the printed z advection filter is the oracle's
    with the slices in reverse order (the 7-point z filter is printed the
    same way): the oracle keeps the +d/dz sign of the x and y filters."""
    G = _golden()
    w, den = N.fe_diffusion_weights(dim)
    gd, gm = G[f"fe{dim}_diffusion"]
    assert den == gd and np.array_equal(_as_array(w, dim).reshape(gm.shape), gm)
    for a, name in enumerate("xyz"[:dim]):
        w, den = N.fe_advection_weights(dim, a)
        gd, gm = G[f"fe{dim}_advection_{name}"]
        m = _as_array(w, dim)
        if dim == 3 and a == 2:
            m = m[::-1]
        assert den == gd and np.array_equal(m.reshape(gm.shape), gm), name


@pytest.mark.parametrize("dim", [2, 3])
def test_filter_moments(dim):
    """Diffusion: zero sum, second moment 2 * den along every axis (so it
    is -d2/da2 on quadratics).  Advection along a: first moment along a
    = den (exact on linear fields), none across."""
    w, den = N.fe_diffusion_weights(dim)
    assert sum(w.values()) == 0
    for a in range(dim):
        assert sum(v * o[a] ** 2 for o, v in w.items()) == -2 * den
        wa, da = N.fe_advection_weights(dim, a)
        for b in range(dim):
            m1 = sum(v * o[b] for o, v in wa.items())
            assert m1 == (da if b == a else 0)


def _coords(g, c):
    """Node coordinates (x, y[, z]) of component c's face grid, as arrays of
    the face shape (index times h; only differences matter)."""
    shp = g.face_shape(c)
    idx = np.indices(shp).astype(np.float64) * g.h
    return [idx[g.dim - 1 - a] for a in range(g.dim)]


def _interior(arr):
    return arr[(slice(2, -2),) * arr.ndim]


def _rate(g, c, Q, U=None, nu=0.0):
    U = U if U is not None else [np.zeros_like(Q) for _ in range(g.dim)]
    gradp = [np.zeros(g.face_shape(k)) for k in range(g.dim)]
    return N.momentum_rate_fe(g, None, c, Q, U, nu, gradp)


@pytest.mark.parametrize("cells,h", [((12, 10), 0.5), ((10, 8, 9), 0.25)])
def test_diffusion_closed_forms(cells, h):
    """In the interior: zero on constants; -f'' on x^2; on x^2 y^2 the
    Laplacian's negative minus h^2 (2D) or 14/13 h^2 (3D): the corner
    weights' signature (the 5-point filter gives no h^2 term)."""
    g = N.MacGrid(cells, h, None)
    for c in range(g.dim):
        X = _coords(g, c)
        r = _rate(g, c, np.full(g.face_shape(c), 3.0), nu=1.0)
        assert np.max(np.abs(_interior(r))) < 1e-12
        for a in range(g.dim):
            r = _rate(g, c, X[a] ** 2, nu=1.0)
            assert np.allclose(_interior(r), -2.0, atol=1e-10)
        x, y = X[0], X[1]
        r = _rate(g, c, x * x * y * y, nu=1.0)
        extra = h * h if g.dim == 2 else 14.0 / 13.0 * h * h
        assert np.allclose(_interior(r), -(2 * x * x + 2 * y * y)[(slice(2, -2),) * g.dim] - extra, atol=1e-10)


@pytest.mark.parametrize("cells,h", [((12, 10), 0.5), ((10, 8, 9), 0.25)])
def test_advection_closed_forms(cells, h):
    """In the interior, with unit advecting velocity along one axis at a
    time: exact on linear fields (each axis's own slope, so a swapped or
    sign-flipped filter fails); on x y^2 (z^2) the (1, 4, 1) smoothing adds
    exactly h^2/3 per smoothed square."""
    g = N.MacGrid(cells, h, None)
    slopes = (2.0, 5.0, -7.0)
    for c in range(g.dim):
        X = _coords(g, c)
        lin = sum(s * X[a] for a, s in zip(range(g.dim), slopes))
        for a in range(g.dim):
            U = [np.zeros_like(lin) for _ in range(g.dim)]
            U[a] = np.ones_like(lin)
            r = _rate(g, c, lin, U)
            assert np.allclose(_interior(r), slopes[a], atol=1e-10), (c, a)
        U = [np.ones_like(lin)] + [np.zeros_like(lin) for _ in range(g.dim - 1)]
        f = X[0] * X[1] ** 2
        want = X[1] ** 2 + h * h / 3.0
        if g.dim == 3:
            f = f * X[2] ** 2
            want = want * (X[2] ** 2 + h * h / 3.0)
        r = _rate(g, c, f, U)
        assert np.allclose(_interior(r), _interior(want), rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_reduces_to_five_point_on_one_axis_fields(dim):
    """A field varying along axis a only, with copy ghosts on every other
    axis: the FE filters equal the 5/7-point filters at every node,
    boundary nodes included (for any advecting velocity and pressure
    gradient)."""
    cells = (9, 7) if dim == 2 else (7, 6, 5)
    g = N.MacGrid(cells, 0.7, None)
    rng = np.random.default_rng(3)
    gradp = [rng.standard_normal(g.face_shape(k)) for k in range(dim)]
    checked = 0
    for c, a in itertools.product(range(dim), range(dim)):
        if any(N.ghost_modes(c, b) != ("copy", "copy") for b in range(dim) if b != a):
            continue
        shp = g.face_shape(c)
        prof = rng.standard_normal(shp[dim - 1 - a])
        bshape = [1] * dim
        bshape[dim - 1 - a] = -1
        Q = np.broadcast_to(prof.reshape(bshape), shp).copy()
        U = [rng.standard_normal(shp) for _ in range(dim)]
        fe = N.momentum_rate_fe(g, None, c, Q, U, 0.3, gradp)
        fp = N.momentum_rate(g, None, c, Q, U, 0.3, gradp)
        assert np.allclose(fe, fp, rtol=1e-12, atol=1e-12), (c, a)
        checked += 1
    assert checked >= dim + 1


@pytest.mark.parametrize("dim", [2, 3])
def test_inflow_ghost_column(dim):
    """A constant tangential component next to the inflow (zero ghost
    column, corner ghosts included): the FE diffusion there is 1/h^2 times
    the constant, hand-worked from the printed weights (2D: (8 - 4)/4; 3D:
    (52 - 26)/26); at the far side, with copy ghosts, it is 0."""
    cells = (6, 5) if dim == 2 else (5, 4, 4)
    h = 0.5
    g = N.MacGrid(cells, h, None)
    c = 1
    Q = np.full(g.face_shape(c), 2.0)
    r = _rate(g, c, Q, nu=1.0)
    x0 = r[(Ellipsis, 0)]
    assert np.allclose(x0, 2.0 / (h * h), rtol=1e-13)
    assert np.max(np.abs(r[(Ellipsis, slice(1, None))])) < 1e-12


@pytest.mark.parametrize("cells", [(16, 8), (8, 8, 8)])
def test_fe_uniform_flow_is_fixed_point(cells):
    """Uniform inflow, no obstacle: the FE momentum step leaves it
    unchanged and the projection does nothing."""
    g = N.MacGrid(cells, 1.0, None)
    q = [np.ones(g.face_shape(0))] + [np.zeros(g.face_shape(c)) for c in range(1, g.dim)]
    qn, pn, dp, qs, b = N.ns_step(g, q, np.zeros(g.shape), 0.1, 0.3, 1.0, fe=True)
    for c in range(g.dim):
        assert np.max(np.abs(qn[c] - q[c])) < 1e-13
    assert np.max(np.abs(pn)) < 1e-13


@pytest.mark.parametrize("cells,block,centre", [((32, 16), 8, (8, 8)), ((16, 8, 8), 4, (4, 4, 4))])
def test_fe_step_is_projected_and_close_to_five_point(cells, block, centre):
    """With the FE filters the step still projects (divergence at the solve
    tolerance) and differs from the 5/7-point step by a small amount (both
    are consistent discretisations of the same operator)."""
    solid = I.block_mask(cells, centre, block)
    g = N.MacGrid(cells, 1.0, solid)
    q = I.ns_initial_velocity(cells, 0, noise=0.05)
    p = np.zeros(g.shape)
    qn, pn, dp, qs, b = N.ns_step(g, q, p, 0.1, 0.3, 1.0, fe=True)
    q5 = N.ns_step(g, q, p, 0.1, 0.3, 1.0)[0]
    fl = ~g.solid
    assert np.linalg.norm(g.divergence(qn)[fl]) <= 1e-10 * np.linalg.norm(g.divergence(qs)[fl])
    for c in range(g.dim):
        d = np.linalg.norm(qn[c] - q5[c]) / np.linalg.norm(q5[c])
        assert 1e-6 < d < 0.05, (c, d)
