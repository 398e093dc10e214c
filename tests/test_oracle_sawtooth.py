"""Pins of the oracle's sawtooth cycle (the paper's own cycle, App. B
recursion) against an independent dense-matrix construction and against
facts that follow from it (no GPU)."""
import numpy as np
import pytest

from oracle import poisson as P
from paper_2402_17913_gb300 import inputs as I


def _fluid_vec(lv, f):
    return f.ravel()[~lv.solid.ravel()]


def _transfer_matrices(fine, coarse):
    """Average restriction (R) and copy prolongation (P) over fluid cells,
    written out cell by cell: a coarse fluid cell takes 1/2^d of each fluid
    child; a fluid child copies its parent."""
    fi, ci = P.fluid_index(fine), P.fluid_index(coarse)
    nf, nc = int((fi >= 0).sum()), int((ci >= 0).sum())
    R, Pm = np.zeros((nc, nf)), np.zeros((nf, nc))
    w = 1.0 / 2 ** fine.dim
    for cell in np.ndindex(*fine.shape):
        if fi[cell] < 0:
            continue
        parent = tuple(c // 2 for c in cell)
        if ci[parent] >= 0:
            R[ci[parent], fi[cell]] = w
            Pm[fi[cell], ci[parent]] = 1.0
    return R, Pm


def _jacobi_matrix_cycle(A, r, post, omega, x):
    d = np.diag(A)
    for _ in range(post):
        x = x + omega * (r - A @ x) / d
    return x


def _case(shape, bc, frac, seed=3):
    rng = np.random.default_rng(seed)
    solid = None
    if frac > 0:
        solid = I.flood_fill_unreachable(rng.random(shape) < frac, bc)
    h = tuple(1.0 / (s + 1) for s in reversed(shape))
    return solid, h


@pytest.mark.parametrize("shape,bc,frac", [((8, 12), (1, 0, 1, 1), 0.1), ((4, 6, 8), (0, 1, 0, 0, 1, 0), 0.05)])
def test_sawtooth_one_level_is_jacobi_from_zero(shape, bc, frac):
    """With a single level the cycle is one Jacobi step from zero, D^-1 r,
    followed by `post` relaxed Jacobi sweeps: (I - w D^-1 A)^post D^-1 r
    in dense-matrix form."""
    solid, h = _case(shape, bc, frac)
    hier = P.build_hierarchy(shape, h, bc, solid, levels=1)
    lv = hier[0]
    A = P.assemble_dense(lv)
    r = (I.blob_rhs(shape, 4) * lv.fluid)
    for post in (0, 1, 3):
        mg = P.Multigrid(hier, post=post, omega=2.0 / 3.0, s=1.0, cycle='sawtooth')
        got = _fluid_vec(lv, mg.precondition(r))
        rv = _fluid_vec(lv, r)
        ref = _jacobi_matrix_cycle(A, rv, post, 2.0 / 3.0, rv / np.diag(A))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("s", [1.0, 0.5])
def test_sawtooth_two_levels_matrix_form(s):
    """Two levels, masked grid with mixed faces: the coarse level gets
    D_1^-1 R r and its own sweeps, the fine level D_0^-1 r + s P x_1 and its
    sweeps (Eqs. r-recur, e19-e23), built from dense A_0, A_1 and explicit
    R, P matrices."""
    shape, bc = (8, 12), (1, 0, 1, 1)
    solid, h = _case(shape, bc, 0.1)
    hier = P.build_hierarchy(shape, h, bc, solid, levels=2)
    f, c = hier
    A0, A1 = P.assemble_dense(f), P.assemble_dense(c)
    R, Pm = _transfer_matrices(f, c)
    r = I.blob_rhs(shape, 5) * f.fluid
    rv = _fluid_vec(f, r)
    post, omega = 2, 2.0 / 3.0
    rc = R @ rv
    x1 = _jacobi_matrix_cycle(A1, rc, post, omega, rc / np.diag(A1))
    x0 = _jacobi_matrix_cycle(A0, rv, post, omega, rv / np.diag(A0) + s * (Pm @ x1))
    mg = P.Multigrid(hier, post=post, omega=omega, s=s, cycle='sawtooth')
    got = _fluid_vec(f, mg.precondition(r))
    assert np.allclose(got, x0, rtol=1e-12, atol=1e-12 * np.abs(x0).max())


def test_sawtooth_is_linear_and_zero_on_solids():
    shape, bc = (16, 16), (0, 0, 0, 0)
    solid, h = _case(shape, bc, 0.08)
    hier = P.build_hierarchy(shape, h, bc, solid)
    mg = P.Multigrid(hier, post=2, s=0.5, cycle='sawtooth')
    r1, r2 = I.blob_rhs(shape, 1) * hier[0].fluid, I.blob_rhs(shape, 2) * hier[0].fluid
    z = mg.precondition(2.0 * r1 - 3.0 * r2)
    assert np.allclose(z, 2.0 * mg.precondition(r1) - 3.0 * mg.precondition(r2), atol=1e-12)
    assert np.all(z[solid] == 0)


def test_sawtooth_stationary_needs_the_halved_correction():
    """As a stationary solver on the 64^2 blob problem the cycle with the
    re-discretised coarse correction (s = 1, twice the Galerkin correction)
    diverges; with s = 1/2 (the Galerkin scaling) every cycle reduces the
    residual."""
    shape = (64, 64)
    h = I.poisson_spacing(shape)
    b = I.blob_rhs(shape, 0)
    hier = P.build_hierarchy(shape, h, (0, 0, 0, 0))
    _, h1 = P.Multigrid(hier, post=2, s=1.0, cycle='sawtooth').stationary(b, 8)
    _, h5 = P.Multigrid(hier, post=2, s=0.5, cycle='sawtooth').stationary(b, 12)
    assert h1[-1] > 10.0
    assert all(b_ < a_ for a_, b_ in zip(h5, h5[1:])) and h5[-1] < 0.25
