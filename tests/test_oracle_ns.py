"""Pins of the FP64 projection-step oracle (Algorithm 1 on a staggered
grid) against invariants and closed forms (no GPU)."""
import numpy as np
import pytest

from oracle import ns as N
from oracle import poisson as P
from paper_2402_17913_gb300 import inputs as I


def _grid(cells, block=None, centre=None):
    solid = None
    if block:
        solid = I.block_mask(cells, centre, block)
    return N.MacGrid(cells, 1.0, solid)


@pytest.mark.parametrize("cells,block,centre", [((16, 8), 4, (6, 4)), ((12, 8, 8), 4, (4, 4, 4))])
def test_minus_div_grad_equals_poisson_operator(cells, block, centre):
    """On the staggered grid -D G equals the pressure operator A_h built by
    the Poisson oracle with the pressure BCs and the solid mask (so the
    projection can reach the solve's tolerance)."""
    g = _grid(cells, block, centre)
    rng = np.random.default_rng(1)
    dp = rng.standard_normal(g.shape) * (~g.solid)
    lhs = -g.divergence(g.gradient(dp)) * (~g.solid)
    rhs = P.apply_A(g.level, dp)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cells", [(16, 8), (8, 8, 8)])
def test_uniform_flow_is_fixed_point(cells):
    """Uniform inflow velocity with no obstacle stays uniform: zero
    divergence, zero pressure correction, momentum leaves it unchanged."""
    g = _grid(cells)
    q = [np.ones(g.face_shape(0))] + [np.zeros(g.face_shape(c)) for c in range(1, g.dim)]
    p = np.zeros(g.shape)
    qn, pn, dp, qs, b = N.ns_step(g, q, p, 0.1, 0.3, 1.0)
    for c in range(g.dim):
        assert np.max(np.abs(qn[c] - q[c])) < 1e-13
    assert np.max(np.abs(pn)) < 1e-13


@pytest.mark.parametrize("cells,block,centre", [((32, 16), 8, (8, 8)), ((16, 8, 8), 4, (4, 4, 4))])
def test_projection_removes_divergence(cells, block, centre):
    """After step 3 of Alg. 1, ||D q||_fluid / ||D q*||_fluid is at the
    relative residual of the pressure solve (1e-12 here)."""
    g = _grid(cells, block, centre)
    q = I.ns_initial_velocity(cells, 0, noise=0.05)
    p = np.zeros(g.shape)
    qn, pn, dp, qs, b = N.ns_step(g, q, p, 0.1, 0.3, 1.0)
    fl = ~g.solid
    d_star = np.linalg.norm(g.divergence(qs)[fl])
    d_new = np.linalg.norm(g.divergence(qn)[fl])
    assert d_star > 1e-3
    assert d_new <= 1e-10 * d_star
    assert np.allclose(pn, dp)
    assert np.all(dp[g.solid] == 0)


def test_pure_diffusion_mode_decays_by_predictor_corrector_factor():
    """With zero inflow and u = 0, a tiny v-mode that is an eigenvector of
    the padded diffusion filter (sin along the walls' normal, the mixed
    zero/copy padding mode along x) is multiplied by 1 - a + a^2 / 2,
    a = nu dt lambda, the amplification of the two-pass scheme of Sec. 2.1
    (Eq. pred-corr-adv-diff) applied to diffusion only."""
    nx, ny = 16, 12
    g = _grid((nx, ny))
    eps = 1e-9     # the self-advection term is O(eps^2): 1e-9 relative
    k, m = 2, 3
    theta = (2 * k - 1) * np.pi / (2 * nx + 1)
    ix = np.arange(nx)
    jy = np.arange(ny + 1)
    mode = np.sin(m * np.pi * jy / ny)[:, None] * np.sin((ix + 1) * theta)[None, :]
    lam = 4 * np.sin(m * np.pi / (2 * ny)) ** 2 + 4 * np.sin(theta / 2) ** 2
    q = [np.zeros(g.face_shape(0)), eps * mode]
    dt, nu = 0.1, 0.7
    qs = N.momentum(g, q, np.zeros(g.shape), dt, nu, 0.0)
    a = nu * dt * lam
    expect = (1 - a + a * a / 2) * eps * mode
    assert np.max(np.abs(qs[1] - expect)) < 1e-8 * eps
    assert np.max(np.abs(qs[0])) < 1e-8 * eps


def test_central_advection_of_linear_field():
    """u = 1 everywhere, nu = 0, v linear in x: in the interior the central
    filter is exact and the two-pass update is v - dt * u * dv/dx.  Faces
    within two of a boundary feel the ghost values through the predictor, so
    the check covers rows 3 .. ny-3 and columns 2 .. nx-3."""
    nx, ny = 12, 10
    g = _grid((nx, ny))
    eps = 1e-3
    xc = (np.arange(nx) + 0.5)
    v = np.tile(eps * xc, (ny + 1, 1))
    q = [np.ones(g.face_shape(0)), v]
    dt = 0.1
    qs = N.momentum(g, q, np.zeros(g.shape), dt, 0.0, 1.0)
    inner = qs[1][3:ny - 2, 2:nx - 2]
    assert np.allclose(inner, v[3:ny - 2, 2:nx - 2] - dt * eps, rtol=0, atol=1e-15)
    assert np.allclose(qs[0], 1.0, atol=1e-15)


def test_solid_faces_are_absorbed():
    """Faces touching the block get the implicit absorption sigma = 1e8:
    their velocity after momentum is ~0 (Eq. Tn+1 entrywise division)."""
    cells = (32, 16)
    g = _grid(cells, 8, (10, 8))
    q = I.ns_initial_velocity(cells, 3)
    qs = N.momentum(g, q, np.zeros(g.shape), 0.1, 0.64, 1.0)
    for c in range(2):
        sf = g.solid_face(c) & ~g.fixed_faces(c)
        assert np.max(np.abs(qs[c][sf])) < 1e-6
