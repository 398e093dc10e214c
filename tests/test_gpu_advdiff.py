"""GPU parity of the implicit advection-diffusion multigrid (one
backward-Euler step, Sec. 2.2 operator, Sec. 3.2 solver) against the FP64
oracle, through the C ABI: one cycle elementwise (the cycle runs in
float32 on a float-float residual, so the bound is a few float32 ulps of the
correction times the cycle's depth), full solves against the dense answer,
and the paper's L1 gauge."""
import numpy as np
import pytest

from oracle import advdiff as A
from paper_2402_17913_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E3 = dict(h=1.0, dt=50.0, nu=2.0, u=1.0, v=1.0)  # Sec. 3.2: C = 50


@pytest.fixture(scope="module")
def L():
    from paper_2402_17913_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def make(L, shape, cycle, coarse, scheme, pre=2, post=2, omega=2 / 3, s=1.0, max_cycles=1000, p=E3):
    opt = L.ad_default_options(cycle=L.MG_CYCLE_SAWTOOTH if cycle == "sawtooth" else L.MG_CYCLE_V, pre=pre,
                               post=post, omega=omega, coarse_scale=s, max_cycles=max_cycles,
                               coarse_op=L.AD_COARSE_GALERKIN if coarse == "galerkin" else L.AD_COARSE_REDISCRETISE)
    hd = L.ad_create((shape[1], shape[0]), p["h"], p["dt"], p["nu"], p["u"], p["v"],
                     L.AD_CENTRAL if scheme == "central" else L.AD_UPWIND, opt)
    hier = A.build_hierarchy(shape, p["h"], p["dt"], p["nu"], p["u"], p["v"], scheme, coarse,
                             levels=L.ad_num_levels(hd))
    mg = A.ADMultigrid(hier, cycle, pre if cycle == "V" else 0, post, omega, s)
    return hd, mg


CASES = [
    # (array shape [y, x], cycle, coarse levels, advection scheme)
    ((128, 128), "V", "rediscretise", "upwind"),
    ((128, 128), "sawtooth", "rediscretise", "upwind"),
    ((40, 96), "V", "galerkin", "central"),       # ragged against the 64 x 16 tiles
    ((64, 256), "sawtooth", "galerkin", "upwind"),
    ((1024, 1024), "V", "rediscretise", "upwind"),  # six tile levels
]


@pytest.mark.parametrize("shape,cycle,coarse,scheme", CASES)
def test_one_cycle_matches_oracle(L, shape, cycle, coarse, scheme):
    """x1 = x0 + M (b - A x0) for one cycle from a random x0 against the
    oracle's cycle on the residual of the same x0 (float64 there)."""
    post, omega, s = (1, 1.0, 0.5) if cycle == "sawtooth" else (2, 2 / 3, 1.0)
    hd, mg = make(L, shape, cycle, coarse, scheme, post=post, omega=omega, s=s, max_cycles=1)
    try:
        rng = np.random.default_rng(3)
        b = I.advdiff_gaussian(shape, gamma=shape[1] / 12.0).astype(np.float32)
        x0 = (0.3 * rng.standard_normal(shape)).astype(np.float32)
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        status, st = L.ad_solve(hd, dev(b), x, rel_tol=0.0, l1_tol=0.0, x0=dev(x0))
        assert status == L.MG_NOT_CONVERGED and st["cycles"] == 1, st
        b64, x064 = b.astype(np.float64), x0.astype(np.float64)
        z = mg.precondition(A.residual(mg.hier[0], b64, x064))
        got = x.cpu().numpy().astype(np.float64) - x064
        err = np.linalg.norm(got - z) / np.linalg.norm(z)
        assert err <= 2e-5, err
        assert st["l1_last"] == pytest.approx(np.abs(z).sum(), rel=1e-4)
        assert st["relres"] == pytest.approx(A.relres(mg.hier[0], b64, x064 + z), rel=1e-3)
    finally:
        L.ad_destroy(hd)


@pytest.mark.parametrize("coarse", ["rediscretise", "galerkin"])
def test_solve_reaches_dense_answer(L, coarse):
    """The Sec. 3.2 test (128^2, upwind, C = 50, Gaussian of width 10) by
    V(2,2) cycles to relres 1e-6: the dense solution within the tolerance,
    the oracle's cycle count."""
    shape = (128, 128)
    hd, mg = make(L, shape, "V", coarse, "upwind")
    try:
        b = I.advdiff_gaussian(shape).astype(np.float32)
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        status, st = L.ad_solve(hd, dev(b), x, rel_tol=1e-6)
        assert status == L.MG_OK and st["relres"] <= 1e-6, st
        b64 = b.astype(np.float64)
        ref = A.dense_solve(mg.hier[0], b64)
        xg = x.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(xg - ref) <= 1e-5 * np.linalg.norm(ref)
        _, k, rr, _ = mg.solve(b64, tol=1e-6)
        assert abs(st["cycles"] - k) <= 1, (st["cycles"], k)
        assert st["relres0"] == pytest.approx(rr[0], rel=1e-6)
    finally:
        L.ad_destroy(hd)


def test_paper_form_l1_gauge(L):
    """The paper's form: sawtooth, Jacobi alpha = 1, one sweep, halved coarse
    correction, started from T^n, stopped when the L1 change of one cycle
    is <= 1e-5 (Sec. 3.2): the oracle's cycle count (+-1), and more than
    three orders of L1 reduction in the first 50 cycles."""
    shape = (128, 128)
    hd, mg = make(L, shape, "sawtooth", "rediscretise", "upwind", post=1, omega=1.0, s=0.5, max_cycles=2000)
    try:
        b = I.advdiff_gaussian(shape).astype(np.float32)
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        status, st = L.ad_solve(hd, dev(b), x, rel_tol=0.0, l1_tol=1e-5)
        assert status == L.MG_OK, st
        _, k, _, l1 = mg.solve(b.astype(np.float64), tol=0.0, l1_tol=1e-5, max_cycles=2000)
        assert abs(st["cycles"] - k) <= 1, (st["cycles"], k)
        assert st["l1_first"] == pytest.approx(l1[0], rel=1e-4)
        hd2, _ = make(L, shape, "sawtooth", "rediscretise", "upwind", post=1, omega=1.0, s=0.5, max_cycles=50)
        try:
            _, st50 = L.ad_solve(hd2, dev(b), x, rel_tol=0.0, l1_tol=0.0)
            assert st50["cycles"] == 50 and st50["l1_last"] < 1e-3 * st50["l1_first"], st50
        finally:
            L.ad_destroy(hd2)
    finally:
        L.ad_destroy(hd)


@pytest.mark.parametrize("u,v,nu,scheme", [(-1.0, 0.5, 0.0, "upwind"), (0.7, -1.0, 0.3, "upwind"),
                                           (1.0, 1.0, 2.0, "central")])
def test_other_velocities_and_schemes_solve(L, u, v, nu, scheme):
    """Velocities along -x or -y (the upwind filter mirrored), pure advection
    (nu = 0) and central advection: V(2,2) cycles reach relres 1e-6 and the
    dense answer on a 64 x 96 grid."""
    shape = (64, 96)
    p = dict(h=1.0, dt=4.0, nu=nu, u=u, v=v)
    hd, mg = make(L, shape, "V", "rediscretise", scheme, p=p)
    try:
        b = I.advdiff_gaussian(shape, gamma=6.0, centre=(-10.0, 5.0)).astype(np.float32)
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        status, st = L.ad_solve(hd, dev(b), x, rel_tol=1e-6)
        assert status == L.MG_OK and st["relres"] <= 1e-6, st
        ref = A.dense_solve(mg.hier[0], b.astype(np.float64))
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    finally:
        L.ad_destroy(hd)


def test_divergent_stationary_sawtooth_is_reported(L):
    """The stationary sawtooth with the plain coarse correction diverges on
    the Sec. 3.2 test (oracle pin); the GPU stops with MG_DIVERGED once the
    residual has grown 1000-fold and returns a finite status record."""
    shape = (128, 128)
    hd, mg = make(L, shape, "sawtooth", "rediscretise", "upwind", post=1, omega=1.0, s=1.0, max_cycles=500)
    try:
        b = I.advdiff_gaussian(shape).astype(np.float32)
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        status, st = L.ad_solve(hd, dev(b), x, rel_tol=1e-6)
        assert status == L.MG_DIVERGED and st["cycles"] < 500, st
        _, _, rr, _ = mg.solve(b.astype(np.float64), tol=0.0, max_cycles=st["cycles"])
        assert rr[-1] > 1e3 * rr[0]
    finally:
        L.ad_destroy(hd)
