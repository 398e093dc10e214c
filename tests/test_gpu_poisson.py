"""GPU parity of the multigrid Poisson path against the FP64 oracle, through
the C ABI.  Tolerances: single float32 kernels are compared elementwise to
~1e-5 of the field's scale (a few float32 ulps times the stencil growth);
whole solves must reach relres <= 1e-6 (float64 iterate, checked here with
the oracle's operator) and relative L2 error <= 1e-5 against x*."""
import ctypes

import numpy as np
import pytest

from oracle import poisson as P
from paper_2402_17913_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2402_17913_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def np_shape(xyz):
    return tuple(reversed(xyz))


CASES = [
    # (numpy shape [y,x] / [z,y,x], bc, solid fraction)
    ((64, 64), (0, 0, 0, 0), 0.0),
    ((48, 96), (1, 0, 1, 1), 0.08),        # ragged tiles along x, mixed BCs, masked
    ((32, 32, 32), (0,) * 6, 0.0),
    ((16, 24, 40), (1, 0, 1, 1, 0, 1), 0.06),
    ((40, 40, 136), (0, 1, 0, 0, 1, 0), 0.05),  # several x/y tiles and z-runs, ragged tails in x and y
]


def make_case(shape, bc, frac, seed=5):
    rng = np.random.default_rng(seed)
    solid = None
    if frac > 0:
        solid = I.flood_fill_unreachable(rng.random(shape) < frac, bc)
    h = tuple(1.0 / (s + 1) for s in reversed(shape))
    return solid, h


def create(L, shape, bc, solid, h, **opt):
    o = L.default_options(**opt)
    st = None if solid is None else dev(solid.astype(np.uint8))
    hdl = L.mg_create(len(shape), tuple(reversed(shape)), h, bc, st, o)
    return hdl


@pytest.mark.parametrize("shape,bc,frac", CASES)
def test_building_blocks_match_oracle(L, shape, bc, frac):
    """Operator, Jacobi sweeps, residual+restriction and prolongation+
    correction on every level, float32 vs the float64 oracle."""
    solid, h = make_case(shape, bc, frac)
    hdl = create(L, shape, bc, solid, h)
    try:
        nl = L.mg_num_levels(hdl)
        hier = P.build_hierarchy(shape, h, bc, solid, levels=nl)
        c = h[0] ** 2
        rng = np.random.default_rng(11)
        for k in range(nl):
            lv = hier[k]
            assert np_shape(L.mg_level_shape(hdl, k)[:len(shape)]) == lv.shape
            x = (rng.standard_normal(lv.shape) * lv.fluid).astype(np.float32)
            b = (rng.standard_normal(lv.shape) * lv.fluid).astype(np.float32)
            x64, b64 = x.astype(np.float64), b.astype(np.float64)
            # operator
            y = torch.zeros(lv.shape, dtype=torch.float32, device="cuda")
            L.mg_apply_operator(hdl, k, dev(x), y)
            ref = c * P.apply_A(lv, x64)
            scale = np.abs(c * lv.diag).max() * np.abs(x64).max()
            assert np.max(np.abs(y.cpu().numpy() - ref)) <= 2e-6 * scale
            # two Jacobi sweeps (A' x = b with b scaled like A')
            bs = (b64 * np.abs(c * lv.diag).max()).astype(np.float32)
            xt = dev(x)
            L.mg_smooth(hdl, k, xt, dev(bs), 2)
            ref = x64
            for _ in range(2):
                ref = P.jacobi(lv, ref, bs.astype(np.float64) / c, 2.0 / 3.0)
            assert np.max(np.abs(xt.cpu().numpy() - ref)) <= 1e-5 * max(np.abs(ref).max(), 1.0)
            if k + 1 < nl:
                co = hier[k + 1]
                bc_t = torch.zeros(co.shape, dtype=torch.float32, device="cuda")
                L.mg_residual_restrict(hdl, k, dev(x), dev(bs), bc_t)
                ref = P.restrict(P.residual(lv, bs.astype(np.float64) / c, x64)) * c
                assert np.max(np.abs(bc_t.cpu().numpy() - ref)) <= 2e-6 * np.abs(bs).max() * 4
                e = (rng.standard_normal(co.shape) * co.fluid).astype(np.float32)
                xt = dev(x)
                L.mg_prolong_correct(hdl, k, dev(e), xt)
                ref = x64 * lv.fluid + 1.0 * P.prolong(e.astype(np.float64), lv)
                assert np.max(np.abs(xt.cpu().numpy() - ref)) <= 1e-6 * (np.abs(ref).max() + 1)
    finally:
        L.mg_destroy(hdl)


@pytest.mark.parametrize("shape,bc,frac", CASES)
def test_one_cycle_matches_oracle(L, shape, bc, frac):
    """One preconditioner cycle (V(2,2), omega 2/3, exact coarsest solve)
    equals the oracle's cycle; the GPU works on A' = h_0x^2 A_h, so
    z_gpu = z_oracle / h_0x^2."""
    solid, h = make_case(shape, bc, frac)
    hdl = create(L, shape, bc, solid, h)
    try:
        nl = L.mg_num_levels(hdl)
        mg = P.Multigrid(P.build_hierarchy(shape, h, bc, solid, levels=nl), s=1.0)
        r = I.blob_rhs(shape, 3, solid=solid).astype(np.float32)
        z = torch.zeros(shape, dtype=torch.float32, device="cuda")
        L.mg_precondition(hdl, dev(r), z)
        ref = mg.precondition(r.astype(np.float64)) / h[0] ** 2
        err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 2e-5, err
    finally:
        L.mg_destroy(hdl)


def solve_and_check(L, shape, bc, solid, h, b, tol=1e-6, relerr=1e-5, **opt):
    hdl = create(L, shape, bc, solid, h, **opt)
    try:
        bt = dev(b)
        xt = torch.zeros_like(bt)
        status, st = L.mg_solve(hdl, bt, xt, tol)
        x64 = torch.zeros(shape, dtype=torch.float64, device="cuda")
        L.mg_get_solution_f64(hdl, x64)
        x64 = x64.cpu().numpy()
        x32 = xt.cpu().numpy()
    finally:
        L.mg_destroy(hdl)
    assert status == L.MG_OK, st
    lv = P.Level(shape, h, bc, solid)
    b64 = b.astype(np.float64)
    rr = P.relres(lv, b64, x64)
    assert rr <= tol, (rr, st)
    assert abs(rr - st["relres"]) <= 1e-3 * tol + 1e-3 * rr
    xs = P.solve_reference(shape, h, bc, b64, solid, tol=1e-12, s=1.0)
    e64 = np.linalg.norm(x64 - xs) / np.linalg.norm(xs)
    e32 = np.linalg.norm(x32 - xs) / np.linalg.norm(xs)
    assert e64 <= relerr and e32 <= relerr, (e64, e32)
    assert np.all(x32[solid] == 0) if solid is not None else True
    return st


@pytest.mark.parametrize("shape,bc,frac", CASES)
def test_solve_matches_oracle(L, shape, bc, frac):
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 0, solid=solid).astype(np.float32)
    solve_and_check(L, shape, bc, solid, h, b)


@pytest.mark.parametrize("shape,bc,frac", CASES)
def test_streaming_kernels_on_every_level(L, shape, bc, frac, monkeypatch):
    """The 2D warp and 3D row-warp level kernels, which the default
    thresholds keep for large levels (>= 2^19 / 2^15 cells), forced onto
    every eligible level and, in 3D, onto the split (column, plane)
    schedule: one cycle and full solves (float32 and FP16 level storage)
    match the oracle with the bounds above, and so does one sawtooth cycle
    (whose up legs run on these kernels)."""
    monkeypatch.setenv("NPMG_STREAM2D_MIN", "0")
    monkeypatch.setenv("NPMG_ROWS3D_MIN", "0")
    monkeypatch.setenv("NPMG_ROWS3D_SPLIT", "2")
    monkeypatch.setenv("NPMG_NO_TMA3D", "1")  # the row-warp kernels, not the TMA-fed ones
    test_one_cycle_matches_oracle(L, shape, bc, frac)
    test_sawtooth_cycle_matches_oracle(L, shape, bc, frac)
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 2, solid=solid).astype(np.float32)
    solve_and_check(L, shape, bc, solid, h, b)
    solve_and_check(L, shape, bc, solid, h, b, prec=1)


T3_CASES = [
    ((32, 32, 32), (0,) * 6, 0.0),
    ((16, 24, 144), (1, 0, 1, 1, 0, 1), 0.06),   # a second, mostly empty 128-wide strip; rows ragged vs 16
    ((40, 40, 160), (0, 1, 0, 0, 1, 0), 0.05),   # several strips, tiles and z-runs
    ((64, 48, 64), (0, 0, 0, 0, 1, 1), 0.0),     # Neumann z faces: the plane link counts 1 and 2
]


@pytest.mark.parametrize("shape,bc,frac", T3_CASES)
def test_tma3d_kernels_on_every_level(L, shape, bc, frac, monkeypatch):
    """The TMA-fed 3D level kernels (plane loads into an mbarrier ring, one
    block barrier per plane), which the default threshold keeps for levels
    of >= 2^15 cells, forced onto every eligible level: one V cycle and one
    sawtooth cycle match the oracle, and full solves with float32, FP16 and
    BF16 level storage reach relres 1e-6 within 1e-5 of x*."""
    monkeypatch.setenv("NPMG_TMA3D_MIN", "0")
    test_one_cycle_matches_oracle(L, shape, bc, frac)
    test_sawtooth_cycle_matches_oracle(L, shape, bc, frac)
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 2, solid=solid).astype(np.float32)
    its = [solve_and_check(L, shape, bc, solid, h, b, prec=prec)["iters"] for prec in (0, 1, 2)]
    # the CG direction update on the TMA-fed kernel (the default with these
    # level kernels) and on the marching kernel: the same iterations
    monkeypatch.setenv("NPMG_NO_TMA3D_CG", "1")
    st = solve_and_check(L, shape, bc, solid, h, b)
    assert abs(st["iters"] - its[0]) <= 1, (st["iters"], its)


CLUSTER_CASES = [
    ((256, 256), (0, 0, 0, 0), 0.0, None),
    ((256, 512), (1, 0, 1, 1), 0.05, None),   # masked, mixed faces
    ((128, 384), (0, 1, 0, 0), 0.08, None),   # rows of 48 and 24 cells per group pass
    ((256, 256), (0, 0, 0, 0), 0.0, "16"),    # coarse cycle from the deepest distributable level
    ((512, 256), (1, 0, 1, 1), 0.05, "8192"),  # coarse cycle from the single-block kernel's first level
]


def _cycle_launches(L, shape, bc, solid, h):
    hdl = create(L, shape, bc, solid, h)
    try:
        r = torch.ones(shape, dtype=torch.float32, device="cuda")
        z = torch.zeros(shape, dtype=torch.float32, device="cuda")
        n0 = L.mg_kernel_launches(hdl)
        L.mg_precondition(hdl, r, z)
        torch.cuda.synchronize()
        return L.mg_kernel_launches(hdl) - n0
    finally:
        L.mg_destroy(hdl)


@pytest.mark.parametrize("shape,bc,frac,coarse", CLUSTER_CASES)
def test_cluster_middle_levels_match_oracle(L, shape, bc, frac, coarse, monkeypatch):
    """With NPMG_CLUSTER2D=1, 2D float32 V(2,2) cycles run their middle
    levels and the coarse cycle in one thread-block cluster launch (fewer
    launches per cycle than the legs launched one by one): one cycle equals
    the oracle's, full solves reach relres 1e-6 within 1e-5 of x*, and with
    the cluster path off the solve takes the same iterations."""
    if coarse:
        monkeypatch.setenv("NPMG_CLUSTER_COARSE_CELLS", coarse)
    monkeypatch.setenv("NPMG_CLUSTER2D", "1")
    solid, h = make_case(shape, bc, frac)
    n_cl = _cycle_launches(L, shape, bc, solid, h)
    test_one_cycle_matches_oracle(L, shape, bc, frac)
    b = I.blob_rhs(shape, 6, solid=solid).astype(np.float32)
    st = solve_and_check(L, shape, bc, solid, h, b)
    monkeypatch.setenv("NPMG_CLUSTER2D", "0")
    n_legs = _cycle_launches(L, shape, bc, solid, h)
    assert n_cl < n_legs, (n_cl, n_legs)
    st0 = solve_and_check(L, shape, bc, solid, h, b)
    assert abs(st["iters"] - st0["iters"]) <= 1 and st["outer"] == st0["outer"], (st, st0)


WHOLE_CASES = [
    ((256, 256), (0, 0, 0, 0), 0.0),     # config 1's grid
    ((128, 384), (1, 0, 1, 1), 0.06),    # masked, mixed faces, rows of 96 groups
    ((64, 64), (0, 1, 0, 0), 0.0),
    ((48, 96), (0, 0, 1, 1), 0.08),      # 48 rows: a cluster of 8 blocks, level 0 alone distributed
]


def _solve_launches(L, shape, bc, solid, h, b):
    hdl = create(L, shape, bc, solid, h)
    try:
        bt = dev(b)
        xt = torch.zeros_like(bt)
        n0 = L.mg_kernel_launches(hdl)
        status, st = L.mg_solve(hdl, bt, xt, 1e-6)
        return status, st, L.mg_kernel_launches(hdl) - n0, xt.cpu().numpy()
    finally:
        L.mg_destroy(hdl)


@pytest.mark.parametrize("shape,bc,frac", WHOLE_CASES)
def test_cluster_whole_solve_matches_oracle(L, shape, bc, frac, monkeypatch):
    """A small 2D grid runs each inner CG solve in one thread-block-cluster
    launch (the float64 refinement steps between them on all SMs): relres
    1e-6 within 1e-5 of the converged
    oracle, the CG iterations (within 1 or 3%) and refinement steps of the
    kernels launched one by one, a handful of launches per solve, and the
    same bits on a second solve."""
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 4, solid=solid).astype(np.float32)
    st = solve_and_check(L, shape, bc, solid, h, b)
    status, st1, n_cl, x1 = _solve_launches(L, shape, bc, solid, h, b)
    status2, _, _, x2 = _solve_launches(L, shape, bc, solid, h, b)
    assert status == status2 == L.MG_OK and np.array_equal(x1, x2)
    # per refinement step: the cluster launch, the loop's condition kernels,
    # the float64 update and residual
    assert st1["iters"] == st["iters"] and n_cl <= 8 + 6 * st1["outer"], (n_cl, st1)
    monkeypatch.setenv("NPMG_NO_CLUSTER_PCG", "1")
    st0 = solve_and_check(L, shape, bc, solid, h, b)
    _, _, n_legs, _ = _solve_launches(L, shape, bc, solid, h, b)
    # the dot products sum in another order (block sums over the cluster
    # instead of the grid's partials): a solve of 100 iterations may end a
    # few iterations apart
    assert abs(st["iters"] - st0["iters"]) <= max(1, st0["iters"] // 30), (st, st0)
    assert st["outer"] == st0["outer"], (st, st0)
    assert n_legs > 5 * n_cl, (n_legs, n_cl)


def test_cluster_whole_solve_limits(L):
    """In the cluster-launch solve the inner iteration cap ends each inner
    solve and the refinement cap ends the solve: max_inner = 2, max_outer = 1
    gives MG_NOT_CONVERGED after two CG iterations, with the oracle's
    relres after two PCG iterations; a zero right-hand side returns zero
    without iterating."""
    shape = (256, 256)
    h = I.poisson_spacing(shape)
    b32 = I.blob_rhs(shape, 0).astype(np.float32)
    b = dev(b32)
    hdl = create(L, shape, (0, 0, 0, 0), None, h, max_inner=2, max_outer=1)
    try:
        x = torch.zeros_like(b)
        status, st = L.mg_solve(hdl, b, x, 1e-6)
        assert status == L.MG_NOT_CONVERGED and st["iters"] == 2, st
        z = torch.zeros_like(b)
        status0, st0 = L.mg_solve(hdl, z, x, 1e-6)
        assert status0 == L.MG_OK and st0["iters"] == 0 and float(x.abs().max()) == 0.0
    finally:
        L.mg_destroy(hdl)
    mg = P.Multigrid(P.build_hierarchy(shape, h, (0, 0, 0, 0)), s=1.0)
    _, hist, _ = P.pcg(mg, b32.astype(np.float64), tol=1e-6, max_iters=2)
    assert abs(st["relres"] - hist[-1]) <= 1e-4 * hist[-1], (st["relres"], hist)


@pytest.mark.parametrize("shape,bc,frac", CASES)
def test_sawtooth_cycle_matches_oracle(L, shape, bc, frac):
    """One cycle of the paper's sawtooth (App. B recursion; omega 2/3, two
    post sweeps, coarse scale 1/2) equals the oracle's sawtooth cycle, up to
    the h_0x^2 scaling of A' (down legs on the tile kernel, up legs on the
    level's fused kernel, as in the V cycle)."""
    solid, h = make_case(shape, bc, frac)
    hdl = create(L, shape, bc, solid, h, cycle=L.MG_CYCLE_SAWTOOTH, coarse_scale=0.5)
    try:
        nl = L.mg_num_levels(hdl)
        mg = P.Multigrid(P.build_hierarchy(shape, h, bc, solid, levels=nl), post=2, s=0.5, cycle='sawtooth')
        r = I.blob_rhs(shape, 3, solid=solid).astype(np.float32)
        z = torch.zeros(shape, dtype=torch.float32, device="cuda")
        L.mg_precondition(hdl, dev(r), z)
        ref = mg.precondition(r.astype(np.float64)) / h[0] ** 2
        err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 2e-5, err
    finally:
        L.mg_destroy(hdl)


def test_sawtooth_stationary_solve(L):
    """The sawtooth as a stationary solver (no CG) with the halved coarse
    correction reaches relres 1e-6 and the converged oracle solution; it
    takes many more cycles than V(2,2)-preconditioned CG."""
    shape = (64, 64)
    h = I.poisson_spacing(shape)
    b = I.blob_rhs(shape, 0).astype(np.float32)
    st = solve_and_check(L, shape, (0, 0, 0, 0), None, h, b, cycle=L.MG_CYCLE_SAWTOOTH, krylov=0,
                         coarse_scale=0.5, max_inner=4000)
    st_v = solve_and_check(L, shape, (0, 0, 0, 0), None, h, b)
    assert st["iters"] > 5 * st_v["iters"], (st["iters"], st_v["iters"])


def test_solve_256_blob_iterations_match_oracle(L):
    """256^2, zero Dirichlet, 8-blob RHS (seed 0), 7 levels: relres 1e-6;
    the refinement loop takes the oracle's number of CG iterations (+-2)."""
    shape = (256, 256)
    h = I.poisson_spacing(shape)
    b = I.blob_rhs(shape, 0).astype(np.float32)
    st = solve_and_check(L, shape, (0, 0, 0, 0), None, h, b)
    assert st["levels"] == 7
    mg = P.Multigrid(P.build_hierarchy(shape, h, (0, 0, 0, 0)), s=1.0)
    _, hist, inner = P.pcg_ir(mg, b.astype(np.float64), tol=1e-6, inner_floor=1e-4)
    assert abs(st["iters"] - inner) <= 2, (st["iters"], inner)
    assert st["outer"] == len(hist) - 1


def test_manufactured_solution_second_order(L):
    """The GPU solution of b = 2 pi^2 sin sin equals the closed form
    (2 pi^2 / lambda_11) v_11 and converges at second order to sin sin."""
    errs = []
    for N in (64, 128, 256):
        shape = (N, N)
        h = I.poisson_spacing(shape)
        b = I.manufactured_rhs(shape).astype(np.float32)
        hdl = create(L, shape, (0, 0, 0, 0), None, h)
        try:
            bt = dev(b)
            xt = torch.zeros_like(bt)
            L.mg_solve(hdl, bt, xt, 1e-10)
            x64 = torch.zeros(shape, dtype=torch.float64, device="cuda")
            L.mg_get_solution_f64(hdl, x64)
            x64 = x64.cpu().numpy()
        finally:
            L.mg_destroy(hdl)
        X = I.node_coords(shape)
        v = np.sin(np.pi * X[0]) * np.sin(np.pi * X[1])
        lam = 2 * 4 / h[0] ** 2 * np.sin(np.pi * h[0] / 2) ** 2
        exact = 2 * np.pi ** 2 / lam * v
        # the RHS was rounded to float32: error bound ~ 1e-7 relative
        assert np.max(np.abs(x64 - exact)) <= 1e-6
        errs.append(np.max(np.abs(x64 - v)))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_reaches_tolerance(L, prec):
    """FP16 / BF16 inner storage with float64 refinement: same relres and
    error bound as float32 (2D masked and 3D)."""
    for shape, bc, frac in (CASES[1], CASES[2]):
        solid, h = make_case(shape, bc, frac)
        b = I.blob_rhs(shape, 1, solid=solid).astype(np.float32)
        st = solve_and_check(L, shape, bc, solid, h, b, prec=prec)
        assert st["outer"] >= 2


def test_stationary_cycle_with_unscaled_correction_diverges(L):
    """krylov = 0 with s = 1: the bare V-cycle diverges (oracle pin); the
    device guard reports MG_DIVERGED instead of looping."""
    shape = (256, 256)
    h = I.poisson_spacing(shape)
    b = dev(I.blob_rhs(shape, 0).astype(np.float32))
    hdl = create(L, shape, (0, 0, 0, 0), None, h, krylov=0, coarse_scale=1.0)
    try:
        x = torch.zeros_like(b)
        status, st = L.mg_solve(hdl, b, x, 1e-6)
    finally:
        L.mg_destroy(hdl)
    assert status == L.MG_DIVERGED, st


def test_stationary_cycle_with_scaled_correction_converges(L):
    """krylov = 0 with s = 0.7 converges (oracle pin: < 0.5 after 6 cycles)."""
    shape = (128, 128)
    h = I.poisson_spacing(shape)
    b = I.blob_rhs(shape, 0).astype(np.float32)
    solve_and_check(L, shape, (0, 0, 0, 0), None, h, b, krylov=0, coarse_scale=0.7)


def test_iteration_limit_reports_not_converged(L):
    """max_inner = 2, max_outer = 1: MG_NOT_CONVERGED with the partial
    iterate, whose relres equals the oracle's after two PCG iterations
    (2.0499: the residual norm of MG-PCG may grow in early iterations)."""
    shape = (128, 128)
    h = I.poisson_spacing(shape)
    b32 = I.blob_rhs(shape, 0).astype(np.float32)
    b = dev(b32)
    hdl = create(L, shape, (0, 0, 0, 0), None, h, max_inner=2, max_outer=1)
    try:
        x = torch.zeros_like(b)
        status, st = L.mg_solve(hdl, b, x, 1e-6)
    finally:
        L.mg_destroy(hdl)
    assert status == L.MG_NOT_CONVERGED
    mg = P.Multigrid(P.build_hierarchy(shape, h, (0, 0, 0, 0)), s=1.0)
    _, hist, _ = P.pcg(mg, b32.astype(np.float64), tol=1e-6, max_iters=2)
    assert abs(st["relres"] - hist[-1]) <= 1e-4 * hist[-1], (st["relres"], hist)


def test_zero_rhs_and_exact_guess(L):
    shape = (64, 64)
    h = I.poisson_spacing(shape)
    hdl = create(L, shape, (0, 0, 0, 0), None, h)
    try:
        b = torch.zeros(shape, dtype=torch.float32, device="cuda")
        x = torch.ones_like(b)
        status, st = L.mg_solve(hdl, b, x, 1e-6)
        assert status == L.MG_OK and st["iters"] == 0
        assert torch.count_nonzero(x).item() == 0
    finally:
        L.mg_destroy(hdl)


def test_repeat_solves_are_deterministic(L):
    shape = (128, 64)
    solid, h = make_case(shape, (1, 0, 1, 1), 0.05)
    b = dev(I.blob_rhs(shape, 4, solid=solid).astype(np.float32))
    hdl = create(L, shape, (1, 0, 1, 1), solid, h)
    try:
        outs = []
        for _ in range(2):
            x = torch.zeros_like(b)
            L.mg_solve(hdl, b, x, 1e-6)
            outs.append(x.clone())
    finally:
        L.mg_destroy(hdl)
    assert torch.equal(outs[0], outs[1])


def test_misaligned_pointer_is_rejected_on_the_host(L):
    """Vector loads need 16-byte aligned arrays: a view at a 4-byte offset
    is rejected with MG_ERR_INVALID before anything is launched."""
    shape = (64, 64)
    h = I.poisson_spacing(shape)
    hdl = create(L, shape, (0, 0, 0, 0), None, h)
    try:
        buf = torch.zeros(64 * 64 + 1, dtype=torch.float32, device="cuda")
        b = buf[1:]
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        import ctypes
        st = L.load().mg_solve(hdl, b.data_ptr(), x.data_ptr(), 1e-6, L.stream_ptr(), None)
        assert st == L.MG_ERR_INVALID
        assert "aligned" in L.last_error()
    finally:
        L.mg_destroy(hdl)


@pytest.mark.parametrize("shape,bc,frac", [CASES[1], CASES[4]])
def test_device_loop_matches_host_loop(L, shape, bc, frac, monkeypatch):
    """The refinement loop run on the device (one graph with conditional
    while nodes) and on the host (a graph launch and a state read per CG
    chunk) launch the same kernels in the same order: the same iterations,
    the same float32 solution bit for bit, and the float-float iterate read
    back from the buffer the device loop left current."""
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 4, solid=solid).astype(np.float32)
    out = []
    for host in (False, True):
        if host:
            monkeypatch.setenv("NPMG_NO_DEVICE_LOOP", "1")
        hdl = create(L, shape, bc, solid, h)
        try:
            x = torch.zeros(shape, dtype=torch.float32, device="cuda")
            runs = []
            for _ in range(2):  # a second solve on the same handle reuses the graphs
                x.zero_()
                status, st = L.mg_solve(hdl, dev(b), x, 1e-6)
                assert status == L.MG_OK and st["relres"] <= 1e-6
                x64 = torch.zeros(shape, dtype=torch.float64, device="cuda")
                L.mg_get_solution_f64(hdl, x64)
                runs.append((st["iters"], st["outer"], x.clone(), x64))
            out.append(runs)
        finally:
            L.mg_destroy(hdl)
    for (it_d, ou_d, x_d, x64_d), (it_h, ou_h, x_h, x64_h) in zip(*out):
        assert (it_d, ou_d) == (it_h, ou_h)
        assert torch.equal(x_d, x_h) and torch.equal(x64_d, x64_h)


def test_building_blocks_reject_misaligned_arrays(L):
    """Every entry point that takes caller arrays refuses a view at a 4-byte
    offset (the kernels move float4 vectors) with MG_ERR_INVALID before it
    enqueues anything: the output arrays are left untouched."""
    shape = (64, 64)
    h = I.poisson_spacing(shape)
    hdl = create(L, shape, (0, 0, 0, 0), None, h)
    lib = L.load()
    s = L.stream_ptr()
    try:
        n = 64 * 64
        buf = torch.full((n + 4,), 7.0, dtype=torch.float32, device="cuda")
        bad = buf[1:n + 1]
        good = torch.full((n,), 7.0, dtype=torch.float32, device="cuda")
        coarse = torch.full((n // 4,), 7.0, dtype=torch.float32, device="cuda")
        calls = {
            "mg_apply_operator": lambda a, c: lib.mg_apply_operator(hdl, 0, a.data_ptr(), c.data_ptr(), s),
            "mg_smooth": lambda a, c: lib.mg_smooth(hdl, 0, c.data_ptr(), a.data_ptr(), 2, s),
            "mg_residual_restrict": lambda a, c: lib.mg_residual_restrict(hdl, 0, a.data_ptr(), a.data_ptr(),
                                                                          coarse.data_ptr(), s),
            "mg_prolong_correct": lambda a, c: lib.mg_prolong_correct(hdl, 0, coarse.data_ptr(), a.data_ptr(), s),
            "mg_precondition": lambda a, c: lib.mg_precondition(hdl, a.data_ptr(), c.data_ptr(), s),
        }
        o = L.default_options()
        calls["mg_vcycle_noalloc"] = lambda a, c: lib.mg_vcycle_noalloc(
            2, L._i64_3(64, 64, 1), L._d3(h[0], h[1], 1.0), L._i6(0, 0, 0, 0, 0, 0), None, ctypes.byref(o),
            a.data_ptr(), c.data_ptr(), s)
        for name, call in calls.items():
            torch.cuda.synchronize()
            st = call(bad, good)
            assert st == L.MG_ERR_INVALID, name
            assert "aligned" in L.last_error(), (name, L.last_error())
            torch.cuda.synchronize()
            assert torch.all(good == 7.0) and torch.all(buf == 7.0) and torch.all(coarse == 7.0), name
    finally:
        L.mg_destroy(hdl)


@pytest.mark.parametrize("shape,bc,frac", [CASES[1], CASES[2]])
def test_float_float_refinement_matches_float64(L, shape, bc, frac):
    """The refinement loop's iterate and outer residual in float64 (the
    default) and in float-float pairs (MG_REFINE_FF): both reach relres 1e-6
    within 1e-5 of x*, with the same refinement steps and CG iterations up
    to one (the two residuals differ only in their last bits), for float32
    and FP16 level storage."""
    solid, h = make_case(shape, bc, frac)
    b = I.blob_rhs(shape, 1, solid=solid).astype(np.float32)
    for prec in (0, 1):
        s64 = solve_and_check(L, shape, bc, solid, h, b, prec=prec)
        sff = solve_and_check(L, shape, bc, solid, h, b, prec=prec, refine=L.MG_REFINE_FF)
        assert abs(s64["iters"] - sff["iters"]) <= 1 and s64["outer"] == sff["outer"], (s64, sff)
