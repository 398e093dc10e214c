"""Pins of the FP64 initial-guess network oracle: brute-force convolution,
adjoint identities of every backward piece, finite-difference gradients,
positive homogeneity, and a hand-worked Adam step (no GPU)."""
import numpy as np
import pytest

from oracle import convnet as C
from paper_2402_17913_gb300 import inputs as I


def test_conv3d_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((27, 3, 2))
    y = C.conv3d(x, w)
    Cin, Z, Y, X = x.shape
    ref = np.zeros((2, Z, Y, X))
    for co in range(2):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    s = 0.0
                    for t, (dz, dy, dx) in enumerate(C.tap_offsets()):
                        zz, y2, x2 = z + dz, yy + dy, xx + dx
                        if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                            s += sum(w[t, ci, co] * x[ci, zz, y2, x2] for ci in range(Cin))
                    ref[co, z, yy, xx] = s
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_backward_pieces_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 4, 8))
    w = rng.standard_normal((27, 4, 3))
    g = rng.standard_normal((3, 6, 4, 8))
    lhs = np.vdot(C.conv3d(x, w), g)
    assert np.isclose(lhs, np.vdot(x, C.conv3d_dgrad(g, w)), rtol=1e-12)
    assert np.isclose(lhs, np.vdot(w, C.conv3d_wgrad(x, g)), rtol=1e-12)
    p = rng.standard_normal((4, 3, 2, 4))
    assert np.isclose(np.vdot(C.pool(x), p), np.vdot(x, C.pool_bwd(p)), rtol=1e-12)
    assert np.isclose(np.vdot(C.up(p), x), np.vdot(p, C.up_bwd(x)), rtol=1e-12)


def test_full_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    W = I.convnet_weights(5)
    x = rng.standard_normal((2, 8, 8, 8))
    t = rng.standard_normal((1, 8, 8, 8))
    y, c = C.forward(W, x)
    dW = C.backward(W, c, y, t)
    eps = 1e-6
    for k in range(C.NLAYERS):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in W[k].shape)
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[k][idx] += eps
            Wm[k][idx] -= eps
            fd = (C.loss(C.forward(Wp, x)[0], t) - C.loss(C.forward(Wm, x)[0], t)) / (2 * eps)
            assert abs(fd - dW[k][idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (k, idx, fd, dW[k][idx])


def test_network_is_positively_homogeneous():
    rng = np.random.default_rng(3)
    W = I.convnet_weights(6)
    x = rng.standard_normal((2, 8, 8, 8))
    y1, _ = C.forward(W, x)
    y2, _ = C.forward(W, 2.5 * x)
    assert np.allclose(y2, 2.5 * y1, rtol=1e-12, atol=1e-14)


def test_adam_step_hand_worked():
    """One step from m = v = 0 with gradient g: m_hat = g, v_hat = g^2, so
    w <- w - lr * g / (|g| + eps)."""
    w = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -4.0])]
    opt = C.Adam(w, lr=0.1)
    w2 = opt.step(w, g)[0]
    assert np.allclose(w2, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 4.0 / (4.0 + 1e-8)], rtol=1e-15)


def test_crop_operator_equals_full_operator_on_interior_cells():
    """On cells whose neighbours all lie in the crop, A_crop is the full
    grid's pressure operator (poisson.Level with the same solid and any
    face types), for h != 1 too."""
    from oracle import poisson as P
    rng = np.random.default_rng(7)
    shape = (10, 12, 14)
    solid = rng.random(shape) < 0.15
    v = rng.standard_normal(shape)
    h = 0.5
    lv = P.Level(shape, (h, h, h), (1, 0, 1, 1, 0, 1), solid)
    full = P.apply_A(lv, v)
    z0, y0, x0 = 2, 3, 4
    crop = (slice(z0, z0 + 6), slice(y0, y0 + 7), slice(x0, x0 + 8))
    got = C.crop_operator(v[crop], ~solid[crop], h)
    inner = C.interior(got.shape)
    assert np.allclose(got[inner], full[crop][inner], rtol=1e-13, atol=1e-12)


def test_crop_operator_is_symmetric_and_kills_constants():
    rng = np.random.default_rng(8)
    shape = (6, 7, 8)
    fluid = rng.random(shape) > 0.2
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    assert np.isclose(np.vdot(C.crop_operator(u, fluid), v), np.vdot(u, C.crop_operator(v, fluid)), rtol=1e-12)
    assert np.allclose(C.crop_operator(np.full(shape, 3.0), fluid), 0.0)


def test_residual_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    shape = (5, 6, 7)
    fluid = rng.random(shape) > 0.2
    y, b = rng.standard_normal(shape), rng.standard_normal(shape)
    loss, g = C.residual_loss(y, b, fluid, h=0.7)
    eps = 1e-6
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in shape)
        yp, ym = y.copy(), y.copy()
        yp[idx] += eps
        ym[idx] -= eps
        fd = (C.residual_loss(yp, b, fluid, 0.7)[0] - C.residual_loss(ym, b, fluid, 0.7)[0]) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-6), (idx, fd, g[idx])
    # the exact solution of the interior equations has zero loss
    r_only_boundary = C.interior(shape) & fluid
    assert loss > 0 and np.all(g[~fluid] == 0) and r_only_boundary.any()


def test_backward_from_matches_backward_for_the_l2_loss():
    rng = np.random.default_rng(10)
    W = I.convnet_weights(3)
    x = rng.standard_normal((2, 8, 8, 8))
    t = rng.standard_normal((1, 8, 8, 8))
    y, c = C.forward(W, x)
    a = C.backward(W, c, y, t)
    b = C.backward_from(W, c, (y - t) / y.size)
    for k in range(C.NLAYERS):
        assert np.array_equal(a[k], b[k])


def test_net_input_scales_each_field_by_its_own_rms():
    rng = np.random.default_rng(11)
    b = rng.standard_normal((8, 8, 8)) * 3.0
    p = rng.standard_normal((8, 8, 8)) * 1e6
    x, rb = C.net_input(b, p)
    assert np.isclose(rb, np.sqrt(np.mean(b * b)), rtol=1e-14)
    assert np.isclose(np.sqrt(np.mean(x[0] ** 2)), 1.0, rtol=1e-13)
    assert np.isclose(np.sqrt(np.mean(x[1] ** 2)), 1.0, rtol=1e-13)
    # the guess rms(b) * net(x) is positively homogeneous in b and ignores
    # the scale of p
    W = I.convnet_weights(4)
    y1 = C.forward(W, C.net_input(b, p)[0])[0] * C.net_input(b, p)[1]
    y2 = C.forward(W, C.net_input(2.0 * b, 7.0 * p)[0])[0] * C.net_input(2.0 * b, 7.0 * p)[1]
    assert np.allclose(y2, 2.0 * y1, rtol=1e-12)
    z, rz = C.net_input(np.zeros_like(b), np.zeros_like(p))
    assert rz == 1.0 and not z.any()


def test_bf16_round_hand_worked_values():
    """Round-to-nearest-even to 8 significant bits: below / above half an
    ulp, exact ties to the even significand (down and up), a carry into the
    exponent, sign, and values already bfloat16 unchanged."""
    x = np.array([1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -7 + 2.0 ** -8,
                  2.0 - 2.0 ** -9, -3.14159265, 0.15625, -0.0])
    want = np.array([1.0, 1.0 + 2.0 ** -7, 1.0, 1.0 + 2.0 ** -6, 2.0, -3.140625, 0.15625, -0.0])
    got = C.bf16_round(x)
    assert np.array_equal(got, want), got
    assert np.array_equal(C.bf16_round(got), got)  # idempotent


def test_bf16_round_error_bound():
    """|round(x) - x| <= (2^-8 + 2^-24) |x|: half an ulp of an 8-bit significand,
    after the rounding to float32 (half an ulp of 24 bits)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)
    r = C.bf16_round(x)
    assert np.all(np.abs(r - x) <= (2.0 ** -8 + 2.0 ** -24) * np.abs(x))
    assert np.max(np.abs(r - x) / np.abs(x)) > 0.9 * 2.0 ** -8  # the bound is reached
    assert np.mean(r != x) > 0.99


def test_rounding_hook_is_the_identity_when_absent_and_bounded_when_bf16():
    """forward/backward with rnd=None are the plain float64 network; with a
    rounding that does nothing they are bit for bit the same; with bfloat16
    storage the output and gradients stay within a few bfloat16 roundings."""
    W = [C.bf16_round(w) for w in I.convnet_weights(21)]
    rng = np.random.default_rng(22)
    x = C.bf16_round(rng.standard_normal((2, 8, 8, 8)))
    t = rng.standard_normal((1, 8, 8, 8))
    y0, c0 = C.forward(W, x)
    y1, c1 = C.forward(W, x, rnd=lambda a: a)
    g0 = C.backward(W, c0, y0, t)
    g1 = C.backward(W, c1, y0, t, rnd=lambda a: a)
    assert np.array_equal(y0, y1.astype(np.float32).astype(np.float64)) or np.allclose(y0, y1, rtol=1e-7)
    for a, b in zip(g0, g1):
        assert np.allclose(a, b, rtol=1e-6, atol=0)
    yb, cb = C.forward(W, x, rnd=C.bf16_round)
    gb = C.backward(W, cb, yb, t, rnd=C.bf16_round)
    assert np.linalg.norm(yb - y0) <= 2e-2 * np.linalg.norm(y0)
    for a, b in zip(g0, gb):
        assert np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(a)
