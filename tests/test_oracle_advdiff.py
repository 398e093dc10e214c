"""Pins of the implicit advection-diffusion oracle (one backward-Euler step
solved by multigrid, Sec. 2.2 and Sec. 3.2) against the printed filters,
closed forms, the dense Galerkin product and the paper's reported
convergence (no GPU)."""
import os

import numpy as np
import pytest
import scipy.fft

from oracle import advdiff as A
from paper_2402_17913_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "advdiff_filters_sec2.txt")


def _golden():
    out, name = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                name = line[1:line.index("]")]
                out[name] = []
            else:
                out[name].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in out.items()}


def _as_matrix(w):
    """Stencil (c, xm, xp, ym, yp) in the printed layout [x][y]."""
    c, xm, xp, ym, yp = w
    m = np.zeros((3, 3))
    m[1, 1], m[0, 1], m[2, 1], m[1, 0], m[1, 2] = c, xm, xp, ym, yp
    return m


@pytest.mark.parametrize("u,v,nu,dt,h", [(1.0, 1.0, 2.0, 50.0, 1.0), (0.3, -0.7, 0.05, 2.0, 0.5)])
def test_central_operator_is_the_printed_sum(u, v, nu, dt, h):
    """Eq. BE-advection-concise: A = identity + u dt/(2 dx) Ax + v dt/(2 dx)
    Ay + nu dt/dx^2 D, with the printed matrices."""
    G = _golden()
    want = (G["identity"] + u * dt / (2 * h) * G["advection_x_central"] + v * dt / (2 * h) * G["advection_y_central"]
            + nu * dt / h ** 2 * G["diffusion"])
    assert np.allclose(_as_matrix(A.stencil(h, dt, nu, u, v, 'central')), want, rtol=1e-14, atol=1e-14)


def test_upwind_operator_and_the_printed_upwind_filter():
    """Eq. A-up prints dt/dx [0 0 0; 0 -2 1; 0 1 0]: forward differences,
    the upwind scheme of a velocity along -x and -y (there the oracle's
    advection part is minus the printed filter: u = -1 times the forward
    difference).  For (u, v) = (1, 1) the oracle takes the backward
    differences: the printed filter point-reflected and negated."""
    G = _golden()["advection_upwind"]
    dt, h = 3.0, 1.0
    base = _as_matrix(A.stencil(h, dt, 0.0, 0.0, 0.0, 'upwind'))
    neg = _as_matrix(A.stencil(h, dt, 0.0, -1.0, -1.0, 'upwind')) - base
    pos = _as_matrix(A.stencil(h, dt, 0.0, 1.0, 1.0, 'upwind')) - base
    assert np.allclose(neg, -dt / h * G)
    assert np.allclose(pos, -dt / h * G[::-1, ::-1])
    # row sums: the advection part annihilates constants (a derivative)
    assert abs(pos.sum()) < 1e-14 and abs(neg.sum()) < 1e-14


@pytest.mark.parametrize("shape", [(12, 16), (9, 14)])
def test_pure_diffusion_step_closed_form(shape):
    """u = v = 0: T^{n+1} = (I + nu dt A_h)^{-1} T^n, diagonal in the sine
    basis of the zero-padded grid: eigenvalues 1 + nu dt (4/h^2)
    (sin^2(i pi / 2(nx+1)) + sin^2(j pi / 2(ny+1)))."""
    h, dt, nu = 0.5, 0.3, 1.7
    rng = np.random.default_rng(0)
    b = rng.standard_normal(shape)
    lv = A.ADLevel(shape, A.stencil(h, dt, nu, 0.0, 0.0, 'upwind'))
    ny, nx = shape
    i = np.arange(1, nx + 1)
    j = np.arange(1, ny + 1)
    lam = (4 / h ** 2) * (np.sin(i * np.pi / (2 * (nx + 1)))[None, :] ** 2
                          + np.sin(j * np.pi / (2 * (ny + 1)))[:, None] ** 2)
    bh = scipy.fft.dstn(b, type=1, norm="ortho")
    want = scipy.fft.idstn(bh / (1 + nu * dt * lam), type=1, norm="ortho")
    assert np.allclose(A.dense_solve(lv, b), want, rtol=1e-12, atol=1e-12)
    assert np.allclose(lv.apply(want), b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("u", [0.8, -1.3])
def test_pure_upwind_advection_step_is_the_recurrence(u):
    """nu = v = 0, upwind: every row is the one-sided recurrence
    (1 + C) T_l - C T_{l-1} = T^n_l (u > 0; mirrored for u < 0), C =
    |u| dt / h, with the zero ghost: solved by a loop."""
    shape, h, dt = (5, 11), 1.0, 2.5
    C = abs(u) * dt / h
    rng = np.random.default_rng(1)
    b = rng.standard_normal(shape)
    want = np.zeros(shape)
    for j in range(shape[0]):
        prev = 0.0
        cols = range(shape[1]) if u > 0 else range(shape[1] - 1, -1, -1)
        for i in cols:
            prev = (b[j, i] + C * prev) / (1 + C)
            want[j, i] = prev
    lv = A.ADLevel(shape, A.stencil(h, dt, 0.0, u, 0.0, 'upwind'))
    assert np.allclose(A.dense_solve(lv, b), want, rtol=1e-12, atol=1e-13)


def _R(shape):
    ny, nx = shape
    R = np.zeros((ny * nx // 4, ny * nx))
    for j in range(ny):
        for i in range(nx):
            R[(j // 2) * (nx // 2) + i // 2, j * nx + i] = 0.25
    return R


@pytest.mark.parametrize("scheme", ["upwind", "central"])
def test_galerkin_coarse_operator_is_R_A_P(scheme):
    """The Galerkin levels equal the dense product R A P of the average
    restriction and the copy prolongation (P = 4 R^T) over three levels,
    boundary rows included; the re-discretised levels differ from it by
    the halved diffusion."""
    shape, h, dt, nu, u, v = (16, 8), 1.0, 5.0, 0.7, 1.0, -0.6
    gal = A.build_hierarchy(shape, h, dt, nu, u, v, scheme, 'galerkin', levels=3)
    red = A.build_hierarchy(shape, h, dt, nu, u, v, scheme, 'rediscretise', levels=3)
    Ak = gal[0].dense()
    for k in range(1, 3):
        R = _R(gal[k - 1].shape)
        Ak = R @ Ak @ (4 * R.T)
        assert np.allclose(Ak, gal[k].dense(), rtol=1e-13, atol=1e-13), k
        assert not np.allclose(Ak, red[k].dense(), rtol=1e-6)


@pytest.mark.parametrize("cycle,coarse,pre,post,omega,s", [
    ("V", "rediscretise", 2, 2, 2 / 3, 1.0), ("V", "galerkin", 2, 2, 2 / 3, 1.0),
    ("sawtooth", "galerkin", 0, 2, 2 / 3, 1.0), ("sawtooth", "rediscretise", 0, 1, 1.0, 0.5)])
def test_multigrid_solves_to_the_dense_answer(cycle, coarse, pre, post, omega, s):
    """The stationary multigrid iteration reaches relres 1e-10 and the dense
    solution on a 32x32 copy of the Sec. 3.2 test (upwind, C = 50)."""
    shape = (32, 32)
    b = I.advdiff_gaussian(shape, gamma=3.0)
    hier = A.build_hierarchy(shape, 1.0, 50.0 / 4, 2.0 / 4, 1.0, 1.0, 'upwind', coarse)
    mg = A.ADMultigrid(hier, cycle, pre, post, omega, s)
    x, k, rr, _ = mg.solve(b, tol=1e-10, max_cycles=400)
    assert rr[-1] <= 1e-10, (k, rr[-5:])
    assert np.allclose(x, A.dense_solve(hier[0], b), rtol=1e-8, atol=1e-10)


def test_cycles_are_linear():
    shape = (16, 16)
    rng = np.random.default_rng(2)
    r1, r2 = rng.standard_normal(shape), rng.standard_normal(shape)
    for cycle in ("V", "sawtooth"):
        hier = A.build_hierarchy(shape, 1.0, 4.0, 0.5, 0.7, 0.2, 'upwind')
        mg = A.ADMultigrid(hier, cycle, 2, 2, 2 / 3, 0.8)
        lhs = mg.precondition(2 * r1 - 3 * r2)
        assert np.allclose(lhs, 2 * mg.precondition(r1) - 3 * mg.precondition(r2), rtol=1e-12, atol=1e-12)


def test_paper_reported_l1_reduction():
    """Sec. 3.2 reports, for 128^2 nodes, (u, v) = (1, 1), nu = 2, dt = 50
    (C = 50), upwind advection, a Gaussian of width 10 at the centre and the
    sawtooth cycle with Jacobi alpha = 1 and one sweep, started from the
    previous time level: the L1 norm of the change between successive
    iterates falls by more than three orders of magnitude in the first 50
    iterations.  With the re-discretised coarse levels and the halved
    coarse correction (the reading the stationary sawtooth needs) the
    oracle's iteration does; with the plain correction it diverges."""
    shape = (128, 128)
    b = I.advdiff_gaussian(shape, gamma=10.0)
    hier = A.build_hierarchy(shape, 1.0, 50.0, 2.0, 1.0, 1.0, 'upwind', 'rediscretise')
    _, _, _, l1 = A.ADMultigrid(hier, 'sawtooth', 0, 1, 1.0, 0.5).solve(b, tol=0.0, max_cycles=50)
    assert len(l1) == 50 and l1[49] < 1e-3 * l1[0], (l1[0], l1[49])
    _, _, rr, _ = A.ADMultigrid(hier, 'sawtooth', 0, 1, 1.0, 1.0).solve(b, tol=0.0, max_cycles=50)
    assert rr[-1] > 1e3 * rr[0]
