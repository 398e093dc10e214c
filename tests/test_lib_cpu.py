"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point declared in include/npmg.h, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_17913_gb300 import build, lib as L
    build.build()
    return L.load()


def declared_functions():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not path.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", path)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b((?:mg|ns|gn|ad)_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2402_17913_gb300 import lib as L
    assert sorted(L.EXPORTED) == declared_functions()


def test_default_options(lib):
    from paper_2402_17913_gb300 import lib as L
    o = L.default_options()
    assert (o.pre, o.post, o.krylov, o.levels, o.prec, o.refine) == (2, 2, 1, 0, 0, L.MG_REFINE_FP64)
    assert abs(o.omega - 2.0 / 3.0) < 1e-15 and o.coarse_scale == 1.0


@pytest.mark.parametrize("dim,shape,bc,why", [
    (4, (8, 8, 8), (0,) * 6, "dim"),
    (2, (1, 8, 1), (0,) * 6, "shape"),
    (2, (8, 8, 1), (0, 0, 7, 0, 0, 0), "bc"),
    (2, (8, 8, 1), (1, 1, 1, 1, 0, 0), "singular"),
])
def test_create_rejects_invalid_arguments(lib, dim, shape, bc, why):
    from paper_2402_17913_gb300 import lib as L
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 3)(*shape)
    sp = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    b6 = (ctypes.c_int * 6)(*bc)
    st = lib.mg_create(ctypes.byref(h), dim, shp, sp, b6, None, None, None)
    assert st == L.MG_ERR_INVALID, why
    assert h.value is None
    assert len(lib.mg_last_error()) > 0


@pytest.mark.parametrize("bad", [dict(pre=9), dict(refine=2), dict(cycle=5)])
def test_create_rejects_bad_options(lib, bad):
    from paper_2402_17913_gb300 import lib as L
    o = L.default_options(**bad)
    h = ctypes.c_void_p()
    st = lib.mg_create(ctypes.byref(h), 2, (ctypes.c_int64 * 3)(8, 8, 1), (ctypes.c_double * 3)(1, 1, 1),
                       (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0), None, ctypes.byref(o), None)
    assert st == L.MG_ERR_INVALID


def test_solve_rejects_null(lib):
    from paper_2402_17913_gb300 import lib as L
    assert lib.mg_solve(None, None, None, 1e-6, None, None) == L.MG_ERR_INVALID
    assert lib.ns_step(None, None, None, None, None, 0.1, 0.1, 1.0, 1e-6, None, None) == L.MG_ERR_INVALID
    assert lib.ns_set_stencils(None, L.NS_STENCIL_FE) == L.MG_ERR_INVALID
    assert lib.ad_solve(None, None, None, None, 1e-6, 0.0, None, None) == L.MG_ERR_INVALID
    assert lib.ad_num_levels(None) == 0 and lib.ad_kernel_launches(None) == 0 and lib.ad_destroy(None) == L.MG_OK


def test_ad_create_rejects_invalid_arguments(lib):
    """Argument checks of ad_create run before any CUDA call."""
    from paper_2402_17913_gb300 import lib as L
    out = ctypes.c_void_p()
    cells = (ctypes.c_int64 * 2)(128, 128)
    o = L.ad_default_options()
    assert lib.ad_create(ctypes.byref(out), cells, 1.0, 0.0, 2.0, 1.0, 1.0, L.AD_UPWIND, ctypes.byref(o),
                         None) == L.MG_ERR_INVALID  # dt = 0
    assert lib.ad_create(ctypes.byref(out), (ctypes.c_int64 * 2)(6, 128), 1.0, 1.0, 2.0, 1.0, 1.0, L.AD_UPWIND,
                         ctypes.byref(o), None) == L.MG_ERR_INVALID  # side < 8
    assert lib.ad_create(ctypes.byref(out), cells, 1.0, 1.0, 2.0, 1.0, 1.0, 7, ctypes.byref(o),
                         None) == L.MG_ERR_INVALID  # scheme
    bad = L.ad_default_options(pre=3)
    assert lib.ad_create(ctypes.byref(out), cells, 1.0, 1.0, 2.0, 1.0, 1.0, L.AD_UPWIND, ctypes.byref(bad),
                         None) == L.MG_ERR_INVALID
    big = L.ad_default_options(levels=2)  # coarsest 64 x 64 > 256 nodes for the dense inverse
    assert lib.ad_create(ctypes.byref(out), cells, 1.0, 1.0, 2.0, 1.0, 1.0, L.AD_UPWIND, ctypes.byref(big),
                         None) == L.MG_ERR_INVALID
    assert not out.value


def test_guess_network_rejects_invalid_arguments(lib):
    """Argument checks of the gn_* entry points run before any device work."""
    from paper_2402_17913_gb300 import lib as L
    vp = ctypes.c_void_p
    cells = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.gn_create(None, None, None) == L.MG_ERR_INVALID
    out = vp()
    assert lib.gn_create(ctypes.byref(out), None, None) == L.MG_ERR_INVALID and not out.value
    assert lib.gn_forward(None, 1, cells, None, None, None, None) == L.MG_ERR_INVALID
    assert lib.gn_gradients(None, 1, cells, None, None, None, None, 0, 1.0, None, None, None) == L.MG_ERR_INVALID
    assert lib.gn_conv3d(None, None, None, 1, cells, 0, None, None) == L.MG_ERR_INVALID
    assert lib.gn_conv3d_wgrad(None, None, None, 1, cells, None, 0, None) == L.MG_ERR_INVALID
    assert lib.gn_train(None, 1, 1, 0, 1e-3, 1, None, None) == L.MG_ERR_INVALID
    assert lib.gn_dataset_size(None) == 0
    assert lib.ns_set_guess(None, None) == L.MG_ERR_INVALID
    assert "ns_set_guess" in L.last_error()


def test_noalloc_rejects_misaligned_arrays_before_any_cuda_call(lib):
    """mg_vcycle_noalloc checks the caller's arrays on the host: a pointer
    that is not 16-byte aligned is refused before the device is touched (the
    fake addresses here are never dereferenced)."""
    from paper_2402_17913_gb300 import lib as L
    shp = (ctypes.c_int64 * 3)(32, 32, 1)
    sp = (ctypes.c_double * 3)(1 / 33, 1 / 33, 1.0)
    b6 = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    o = L.default_options()
    for r, z in ((0x10004, 0x20000), (0x10000, 0x20008)):
        st = lib.mg_vcycle_noalloc(2, shp, sp, b6, None, ctypes.byref(o), r, z, None)
        assert st == L.MG_ERR_INVALID
        assert "aligned" in L.last_error()
