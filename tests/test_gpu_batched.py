"""GPU parity of the batched persistent solver (one cooperative launch for a
batch of uneven 2D instances): every instance against the FP64 oracle and
against the single-grid solver, the autotuner, and the bounded barrier."""
import os

import numpy as np
import pytest

from oracle import poisson as P
from paper_2402_17913_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BC = (0, 0, 0, 0)


@pytest.fixture(scope="module")
def L():
    from paper_2402_17913_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def make_batch(sides, seed=7, with_masks=True):
    rng = np.random.default_rng(seed)
    shapes, spacings, solids, rhs = [], [], [], []
    for k, (nx, ny) in enumerate(sides):
        shape = (ny, nx)
        solid = I.random_solid_mask(shape, rng, 0.08) if (with_masks and k % 2 == 0) else None
        shapes.append((nx, ny))
        spacings.append((1.0 / (nx + 1), 1.0 / (ny + 1)))
        solids.append(solid)
        rhs.append(I.blob_rhs(shape, 100 + k, solid=solid).astype(np.float32))
    return shapes, spacings, solids, rhs


def run_batch(L, shapes, spacings, solids, rhs, tol=1e-6, sweeps=2, tile=(64, 16)):
    masks = [None if s is None else torch.from_numpy(s.astype(np.uint8)).cuda() for s in solids]
    b = L.mg_create_batched(shapes, spacings, BC, masks)
    try:
        L.mg_batched_config(b, tile[0], tile[1], sweeps)
        bt = [torch.from_numpy(r).cuda() for r in rhs]
        xt = [torch.zeros_like(t) for t in bt]
        status, stats = L.mg_solve_batched(b, bt, xt, tol)
        xs = [t.cpu().numpy() for t in xt]
    finally:
        L.mg_destroy_batched(b)
    return status, stats, xs


SIDES = [(64, 64), (128, 64), (96, 96), (64, 128), (128, 128), (256, 64)]


def test_batch_matches_oracle_and_single_grid(L):
    shapes, spacings, solids, rhs = make_batch(SIDES)
    status, stats, xs = run_batch(L, shapes, spacings, solids, rhs)
    assert status == L.MG_OK, [s["status_name"] for s in stats]
    for k, ((nx, ny), h, solid, b, x, st) in enumerate(zip(shapes, spacings, solids, rhs, xs, stats)):
        shape = (ny, nx)
        assert st["relres"] <= 1e-6, (k, st)
        xs_ref = P.solve_reference(shape, h, BC, b.astype(np.float64), solid, tol=1e-12, s=1.0)
        err = np.linalg.norm(x - xs_ref) / np.linalg.norm(xs_ref)
        assert err <= 1e-5, (k, err)
        if solid is not None:
            assert np.all(x[solid] == 0)
        # the same algorithm as the single-grid solver: the same CG iteration
        # count up to float32 rounding drift (the two smoother codes round
        # differently; long, anisotropic solves drift by an iteration or two)
        hdl = L.mg_create(2, (nx, ny), h, BC,
                          None if solid is None else torch.from_numpy(solid.astype(np.uint8)).cuda())
        try:
            bt = torch.from_numpy(b).cuda()
            x1 = torch.zeros_like(bt)
            _, s1 = L.mg_solve(hdl, bt, x1, 1e-6)
        finally:
            L.mg_destroy(hdl)
        assert abs(s1["iters"] - st["iters"]) <= max(1, 0.05 * s1["iters"]), (k, s1["iters"], st["iters"])
        assert s1["outer"] == st["outer"]


@pytest.mark.parametrize("sweeps,tile", [(1, (32, 16)), (3, (128, 8)), (2, (64, 32)), (3, (128, 16))])
def test_other_tiles_and_sweep_depths_converge(L, sweeps, tile):
    shapes, spacings, solids, rhs = make_batch(SIDES[:4], seed=11)
    status, stats, xs = run_batch(L, shapes, spacings, solids, rhs, sweeps=sweeps, tile=tile)
    assert status == L.MG_OK
    for (nx, ny), h, solid, b, x in zip(shapes, spacings, solids, rhs, xs):
        ref = P.solve_reference((ny, nx), h, BC, b.astype(np.float64), solid, tol=1e-12, s=1.0)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("sweeps,tile", [(2, (64, 16)), (3, (32, 16))])
def test_level_widths_off_the_float4_grid_use_the_scalar_tiles(L, sweeps, tile):
    """Instances whose level-1 width is not a multiple of 4 (100 -> 50,
    68 -> 34, 132 -> 66) run that level on the scalar tile path and every
    other level on the float4 path; both must give the oracle's solution."""
    shapes, spacings, solids, rhs = make_batch([(100, 68), (68, 100), (64, 64), (132, 100)], seed=13)
    status, stats, xs = run_batch(L, shapes, spacings, solids, rhs, sweeps=sweeps, tile=tile)
    assert status == L.MG_OK, [s["status_name"] for s in stats]
    for (nx, ny), h, solid, b, x, st in zip(shapes, spacings, solids, rhs, xs, stats):
        assert st["relres"] <= 1e-6, st
        ref = P.solve_reference((ny, nx), h, BC, b.astype(np.float64), solid, tol=1e-12, s=1.0)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-5


def test_autotuner_picks_a_valid_choice_and_caches_it(L, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("NPMG_TUNE_CACHE", str(cache))
    shapes, spacings, solids, rhs = make_batch(SIDES[:3], seed=3)
    masks = [None if s is None else torch.from_numpy(s.astype(np.uint8)).cuda() for s in solids]
    b = L.mg_create_batched(shapes, spacings, BC, masks)
    try:
        bt = [torch.from_numpy(r).cuda() for r in rhs]
        xt = [torch.zeros_like(t) for t in bt]
        tx, ty, sw = L.mg_tune_batched(b, bt, xt, 1e-6)
        assert (tx, ty) in ((64, 16), (32, 16), (128, 8), (64, 32), (128, 16)) and sw in (1, 2, 3)
        xt = [torch.zeros_like(t) for t in bt]
        status, _ = L.mg_solve_batched(b, bt, xt, 1e-6)
        assert status == L.MG_OK
    finally:
        L.mg_destroy_batched(b)
    line = cache.read_text().strip().splitlines()[-1].split()
    assert int(line[1]) in (0, 1, 2, 3, 4) and int(line[2]) == sw


def test_autotuner_candidates_start_from_the_given_guess(L, tmp_path, monkeypatch):
    """Every candidate solve of the tuner starts from the guesses d_x holds
    on entry, so the result it leaves (the last candidate: 128x16 tiles,
    three sweeps) is bit for bit a solve from the same guesses with that
    choice."""
    monkeypatch.setenv("NPMG_TUNE_CACHE", str(tmp_path / "tune.txt"))
    shapes, spacings, solids, rhs = make_batch(SIDES[:3], seed=21)
    masks = [None if s is None else torch.from_numpy(s.astype(np.uint8)).cuda() for s in solids]
    b = L.mg_create_batched(shapes, spacings, BC, masks)
    try:
        bt = [torch.from_numpy(r).cuda() for r in rhs]
        xt = [torch.zeros_like(t) for t in bt]
        L.mg_tune_batched(b, bt, xt, 1e-6)
        tuned = [t.cpu().numpy() for t in xt]
        L.mg_batched_config(b, 128, 16, 3)
        xt = [torch.zeros_like(t) for t in bt]
        status, _ = L.mg_solve_batched(b, bt, xt, 1e-6)
        assert status == L.MG_OK
        for a, c in zip(tuned, xt):
            assert np.array_equal(a, c.cpu().numpy())
    finally:
        L.mg_destroy_batched(b)


def test_caller_arrays_off_16_byte_boundaries(L):
    """Right-hand sides, guesses and outputs that start 4 bytes past a
    16-byte boundary take the cell-by-cell refinement loops instead of the
    float4 ones, with the same solution."""
    shapes, spacings, solids, rhs = make_batch(SIDES[:3], seed=17)
    masks = [None if s is None else torch.from_numpy(s.astype(np.uint8)).cuda() for s in solids]
    b = L.mg_create_batched(shapes, spacings, BC, masks)
    try:
        def view(a):
            buf = torch.zeros(a.size + 1, dtype=torch.float32, device="cuda")
            buf[1:] = torch.from_numpy(a.ravel()).cuda()
            return buf[1:].view(a.shape)
        bt = [view(r) for r in rhs]
        xt = [view(np.zeros_like(r)) for r in rhs]
        assert all(t.data_ptr() % 16 == 4 for t in bt + xt)
        status, stats = L.mg_solve_batched(b, bt, xt, 1e-6)
        assert status == L.MG_OK, [s_["status_name"] for s_ in stats]
        for (nx, ny), h, solid, r, x in zip(shapes, spacings, solids, rhs, xt):
            ref = P.solve_reference((ny, nx), h, BC, r.astype(np.float64), solid, tol=1e-12, s=1.0)
            assert np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    finally:
        L.mg_destroy_batched(b)


def test_withheld_barrier_arrival_times_out(L):
    """One block never arrives at the first grid barrier: the others wait a
    bounded time (0.2 s), the solve returns MG_TIMEOUT, and the next solve on
    the same handle works."""
    shapes, spacings, solids, rhs = make_batch(SIDES[:2], seed=5, with_masks=False)
    b = L.mg_create_batched(shapes, spacings, BC, None)
    try:
        bt = [torch.from_numpy(r).cuda() for r in rhs]
        xt = [torch.zeros_like(t) for t in bt]
        L.mg_batched_config(b, 64, 16, 2, barrier_timeout_s=0.2, withhold_first_arrival=True)
        status, stats = L.mg_solve_batched(b, bt, xt, 1e-6)
        assert status == L.MG_TIMEOUT
        assert all(s["status"] == L.MG_TIMEOUT for s in stats)
        L.mg_batched_config(b, 64, 16, 2, barrier_timeout_s=2.0, withhold_first_arrival=False)
        xt = [torch.zeros_like(t) for t in bt]
        status, stats = L.mg_solve_batched(b, bt, xt, 1e-6)
        assert status == L.MG_OK
    finally:
        L.mg_destroy_batched(b)


def test_repeat_batched_solves_are_deterministic(L):
    shapes, spacings, solids, rhs = make_batch(SIDES[:3], seed=9)
    outs = [run_batch(L, shapes, spacings, solids, rhs)[2] for _ in range(2)]
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
