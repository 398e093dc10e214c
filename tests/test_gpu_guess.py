"""What the trained initial-guess network gains over the zero guess, on a
small 3D flow past a cube: solver-generated pairs, residual-loss training on
the GPU, then projection steps from the network's guess against the same
states from zero.  Both solves still run to the same tolerance (plain
multigrid judges the guess), so the fields agree to the solve tolerance."""
import numpy as np
import pytest

from paper_2402_17913_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CELLS = (64, 32, 32)
CUBE, CENTRE = 8, (16, 16, 16)
NU, DT, UIN, TOL = 0.08, 0.1, 1.0, 1e-6  # Re = U L / nu = 100 on the cube side


@pytest.fixture(scope="module")
def L():
    from paper_2402_17913_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def test_trained_guess_cuts_residual_and_iterations(L):
    solid = I.block_mask(CELLS, CENTRE, CUBE)
    solid_t = torch.from_numpy(solid.astype(np.uint8)).cuda()
    ns = L.ns_create(3, CELLS, 1.0, solid_t)
    g = L.gn_create(I.convnet_weights(0, last_scale=1e-3))
    try:
        q = [torch.from_numpy(a.astype(np.float32)).cuda() for a in I.ns_initial_velocity(CELLS, 0)]
        p = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
        L.gn_dataset_reserve(g, (32, 32, 32), 200, 1.0)
        for _ in range(80):
            L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL, stats=False)
            b_ptr, dp_ptr = L.ns_last_fields(ns)
            L.gn_dataset_add(g, CELLS, b_ptr, p, dp_ptr, solid_t)
        assert L.gn_dataset_size(g) == 160
        losses = L.gn_train(g, 600, 4, 3, 1e-3, L.GN_LOSS_RESIDUAL)
        # 0.5 * relres^2 of a minibatch; the zero guess scores about 0.44
        # (interior fraction of a 32^3 crop / 2)
        assert np.mean(losses[-50:]) < 0.25 * np.mean(losses[:50]), (losses[:5], losses[-5:])
        gains = []
        for _ in range(3):
            state = [t.clone() for t in q] + [p.clone()]
            L.ns_set_guess(ns, g)
            sg_status, sg = L.ns_step(ns, state[0], state[1], state[2], state[3], DT, NU, UIN, TOL)
            L.ns_set_guess(ns, None)
            sz_status, sz = L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL)
            assert sg_status == L.MG_OK and sz_status == L.MG_OK
            assert sg["relres"] <= TOL and sz["relres"] <= TOL
            assert sz["guess_relres"] == pytest.approx(1.0)  # zero guess
            assert not sg["guess_rejected"] and sg["guess_relres"] < 0.6, sg
            assert sg["iters"] <= sz["iters"], (sg["iters"], sz["iters"])
            # same step, same tolerance: the fields agree to the solve's accuracy
            for a, c in zip(state, q + [p]):
                an, cn = a.cpu().numpy(), c.cpu().numpy()
                assert np.linalg.norm(an - cn) <= 1e-4 * max(np.linalg.norm(cn), 1.0)
            gains.append((sg["guess_relres"], sz["iters"] - sg["iters"]))
        assert sum(d for _, d in gains) >= 1, gains
    finally:
        L.gn_destroy(g)
        L.ns_destroy(ns)


def test_guess_worse_than_zero_is_rejected(L):
    """A network whose output is huge (large last-layer weights) gives
    relres >> 1: the solve restarts from zero, reports the rejection and
    converges exactly as the zero-guess solve."""
    solid = I.block_mask(CELLS, CENTRE, CUBE)
    solid_t = torch.from_numpy(solid.astype(np.uint8)).cuda()
    ns = L.ns_create(3, CELLS, 1.0, solid_t)
    g = L.gn_create(I.convnet_weights(5, last_scale=1e3))
    try:
        q = [torch.from_numpy(a.astype(np.float32)).cuda() for a in I.ns_initial_velocity(CELLS, 0)]
        p = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
        for _ in range(3):
            L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL, stats=False)
        state = [t.clone() for t in q] + [p.clone()]
        L.ns_set_guess(ns, g)
        _, sg = L.ns_step(ns, state[0], state[1], state[2], state[3], DT, NU, UIN, TOL)
        L.ns_set_guess(ns, None)
        _, sz = L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL)
        assert sg["guess_rejected"] == 1 and sg["guess_relres"] > 1.0
        assert sg["iters"] == sz["iters"] and sg["relres"] <= TOL
        for a, c in zip(state, q + [p]):
            assert torch.equal(a, c)
    finally:
        L.gn_destroy(g)
        L.ns_destroy(ns)


@pytest.mark.parametrize("level", [1, 2])
def test_coarse_guess_path(L, level):
    """The guess on the coarsened grid: ns_coarse_fields restricts b, p and dp
    by 2x2x2 averages (checked against numpy) and coarsens the solid mask;
    a network trained on those fields seeds ns_step through the trilinear
    interpolation without harming the solve: not rejected, no more
    iterations than from zero, same fields to the solve's accuracy."""
    solid = I.block_mask(CELLS, CENTRE, CUBE)
    solid_t = torch.from_numpy(solid.astype(np.uint8)).cuda()
    ns = L.ns_create(3, CELLS, 1.0, solid_t)
    g = L.gn_create(I.convnet_weights(0, last_scale=1e-3))
    q2 = 1 << level
    cells = tuple(c // q2 for c in CELLS)
    nc = cells[0] * cells[1] * cells[2]
    crop = 32 // q2
    try:
        q = [torch.from_numpy(a.astype(np.float32)).cuda() for a in I.ns_initial_velocity(CELLS, 0)]
        p = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
        co = [torch.empty(nc, device="cuda") for _ in range(3)]
        sc = torch.empty(nc, dtype=torch.uint8, device="cuda")
        L.gn_dataset_reserve(g, (crop,) * 3, 200, float(q2))
        for k in range(60):
            L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL, stats=False)
            L.ns_coarse_fields(ns, level, p, co[0], co[1], co[2], sc)
            if k == 0:
                b_ptr, dp_ptr = L.ns_last_fields(ns)
                fine = [raw_tensor(ptr_, solid.shape) for ptr_ in (b_ptr, dp_ptr)]
                torch.cuda.synchronize()
                for f, c in zip((fine[0], p, fine[1]), co):
                    ref = f.cpu().numpy().astype(np.float64)
                    for _ in range(level):
                        nz_, ny_, nx_ = ref.shape
                        ref = ref.reshape(nz_ // 2, 2, ny_ // 2, 2, nx_ // 2, 2).mean(axis=(1, 3, 5))
                    got = c.cpu().numpy().reshape(ref.shape)
                    assert np.allclose(got, ref, rtol=1e-5, atol=1e-6 * max(np.abs(ref).max(), 1e-30))
                sref = solid.astype(bool)
                for _ in range(level):
                    nz_, ny_, nx_ = sref.shape
                    sref = sref.reshape(nz_ // 2, 2, ny_ // 2, 2, nx_ // 2, 2).all(axis=(1, 3, 5))
                assert np.array_equal(sc.cpu().numpy().reshape(sref.shape) != 0, sref)
            L.gn_dataset_add(g, cells, co[0], co[1], co[2], sc)
        L.gn_train(g, 300, 4, 3, 1e-3, L.GN_LOSS_RESIDUAL)
        for _ in range(2):
            state = [t.clone() for t in q] + [p.clone()]
            L.ns_set_guess_level(ns, g, level)
            sg_status, sg = L.ns_step(ns, state[0], state[1], state[2], state[3], DT, NU, UIN, TOL)
            L.ns_set_guess(ns, None)
            sz_status, sz = L.ns_step(ns, q[0], q[1], q[2], p, DT, NU, UIN, TOL)
            assert sg_status == L.MG_OK and sz_status == L.MG_OK and sg["relres"] <= TOL
            assert not sg["guess_rejected"] and sg["guess_relres"] < 1.0, sg
            assert sg["iters"] <= sz["iters"] + 1, (sg["iters"], sz["iters"])
            for a, c in zip(state, q + [p]):
                an, cn = a.cpu().numpy(), c.cpu().numpy()
                assert np.linalg.norm(an - cn) <= 1e-4 * max(np.linalg.norm(cn), 1.0)
    finally:
        L.gn_destroy(g)
        L.ns_destroy(ns)


def raw_tensor(ptr_, shape):
    """A float32 CUDA tensor viewing device memory owned by the library."""
    n = int(np.prod(shape))

    class _Raw:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr_, False), "version": 3}
    return torch.as_tensor(_Raw(), device="cuda").view(shape)
