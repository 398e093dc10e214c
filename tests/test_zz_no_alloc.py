"""The allocation-free entry point mg_vcycle_noalloc, for callers that cannot
call cudaMalloc (inside a capture they do not own, under a fixed memory
budget, in a loop that must not allocate): its cycle must equal the one of
the handle-based mg_precondition, call after call, although all its
temporaries live in one static device array shared by every call.  This file
is collected last so that a stop-at-first-failure run has already run every
other test."""
import numpy as np
import pytest

from paper_2402_17913_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tolerance of the other float32 cycle tests (tests/test_gpu_poisson.py)
RTOL = 2e-5


@pytest.fixture(scope="module")
def L():
    from paper_2402_17913_gb300 import build, lib
    build.build()
    lib.load()
    return lib


CASES = [
    # (numpy shape, bc, solid fraction, pre/post sweeps)
    ((96, 128), (1, 0, 1, 1), 0.06, 2),
    ((32, 32, 32), (0,) * 6, 0.0, 2),
    ((32, 32), (0, 0, 0, 0), 0.0, 2),            # the whole grid in the single-block coarse kernel
    ((64, 64), (0, 1, 0, 0), 0.05, 1),           # runtime-halo tile kernels (one sweep)
    ((64, 96), (0, 0, 1, 0), 0.0, 3),            # runtime-halo tile kernels (three sweeps)
    ((32, 32, 32), (1, 0, 0, 0, 1, 0), 0.08, 2),  # masked 3D
    ((512, 512), (0, 0, 0, 0), 0.05, 2),         # the cell limit, masked
    ((64, 64, 64), (0,) * 6, 0.0, 2),            # the cell limit, 3D
]


@pytest.mark.parametrize("shape,bc,frac,sweeps", CASES)
def test_noalloc_cycle_matches_handle_cycle_twice(L, shape, bc, frac, sweeps):
    rng = np.random.default_rng(21)
    solid = I.flood_fill_unreachable(rng.random(shape) < frac, bc) if frac > 0 else None
    h = tuple(1.0 / (s + 1) for s in reversed(shape))
    xyz = tuple(reversed(shape))
    sol = None if solid is None else torch.from_numpy(solid.astype(np.uint8)).cuda()
    opt = L.default_options(pre=sweeps, post=sweeps)
    hdl = L.mg_create(len(shape), xyz, h, bc, sol, opt)
    try:
        for call in range(2):  # two calls in a row: leftovers in the static array must not matter
            r = torch.from_numpy(I.blob_rhs(shape, 30 + call, solid=solid).astype(np.float32)).cuda()
            z_ref = torch.zeros_like(r)
            z = torch.full_like(r, float("nan"))
            L.mg_precondition(hdl, r, z_ref)
            L.mg_vcycle_noalloc(len(shape), xyz, h, bc, r, z, solid=sol, options=L.default_options(pre=sweeps,
                                                                                               post=sweeps))
            torch.cuda.synchronize()
            err = (torch.linalg.norm(z.double() - z_ref.double()) / torch.linalg.norm(z_ref.double())).item()
            assert err <= RTOL, (call, err)
    finally:
        L.mg_destroy(hdl)


def test_noalloc_reused_setup_follows_the_geometry(L):
    """An unmasked call reuses the set-up (coarsest inverse, coarse image)
    the previous call left only for the same geometry: a sequence that
    changes shape, spacing, faces and mask between calls, and comes back,
    matches the handle cycle at every call."""
    seq = [((64, 64), (0, 0, 0, 0), None), ((64, 64), (0, 0, 0, 0), None), ((96, 128), (0, 0, 0, 0), None),
           ((64, 64), (0, 0, 0, 0), None), ((64, 64), (0, 1, 0, 0), None), ((64, 64), (0, 0, 0, 0), 0.08),
           ((64, 64), (0, 0, 0, 0), None), ((64, 64), (0, 0, 0, 0), "h")]
    for i, (shape, bc, frac) in enumerate(seq):
        rng = np.random.default_rng(40 + i)
        solid = I.flood_fill_unreachable(rng.random(shape) < frac, bc) if isinstance(frac, float) else None
        h = tuple((0.5 if frac == "h" else 1.0) / (s + 1) for s in reversed(shape))
        xyz = tuple(reversed(shape))
        sol = None if solid is None else torch.from_numpy(solid.astype(np.uint8)).cuda()
        hdl = L.mg_create(len(shape), xyz, h, bc, sol, L.default_options())
        try:
            r = torch.from_numpy(I.blob_rhs(shape, 50 + i, solid=solid).astype(np.float32)).cuda()
            z_ref = torch.zeros_like(r)
            z = torch.full_like(r, float("nan"))
            L.mg_precondition(hdl, r, z_ref)
            L.mg_vcycle_noalloc(len(shape), xyz, h, bc, r, z, solid=sol)
            torch.cuda.synchronize()
            err = (torch.linalg.norm(z.double() - z_ref.double()) / torch.linalg.norm(z_ref.double())).item()
            assert err <= RTOL, (i, shape, bc, frac, err)
        finally:
            L.mg_destroy(hdl)


def test_noalloc_rejects_a_coarsest_level_beyond_the_limit(L):
    """Two levels on 64^2 leave a 32^2 coarsest level (1024 cells > 256)."""
    x = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    with pytest.raises(L.MGError) as e:
        L.mg_vcycle_noalloc(2, (64, 64), (1 / 65, 1 / 65), (0, 0, 0, 0), x, x, options=L.default_options(levels=2))
    assert "coarsest" in str(e.value)


def test_noalloc_rejects_sizes_beyond_the_scratch(L):
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(L.MGError) as e:
        L.mg_vcycle_noalloc(2, (1024, 1024), (1e-3, 1e-3), (0, 0, 0, 0), x, x)
    assert "maximum" in str(e.value)
