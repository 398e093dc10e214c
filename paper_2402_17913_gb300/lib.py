"""ctypes binding of ``libnpmg.so`` (declarations in ``include/npmg.h``).

Argument marshalling only: every function forwards to the C entry point of
the same name.  Device arrays are passed as torch CUDA tensors (or raw
integer pointers); streams default to torch's current stream.  There is no
fallback: if the library is missing, ``load()`` raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpmg.so")

MG_OK, MG_ERR_INVALID, MG_ERR_CUDA, MG_ERR_OOM, MG_NOT_CONVERGED, MG_DIVERGED, MG_TIMEOUT = range(7)
MG_BC_DIRICHLET, MG_BC_NEUMANN = 0, 1
MG_FP32, MG_MIXED_FP16, MG_MIXED_BF16 = 0, 1, 2
MG_CYCLE_V, MG_CYCLE_SAWTOOTH = 0, 1
MG_REFINE_FP64, MG_REFINE_FF = 0, 1
NS_STENCIL_FD, NS_STENCIL_FE = 0, 1
AD_UPWIND, AD_CENTRAL = 0, 1
AD_COARSE_REDISCRETISE, AD_COARSE_GALERKIN = 0, 1

STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID", 2: "MG_ERR_CUDA", 3: "MG_ERR_OOM",
                4: "MG_NOT_CONVERGED", 5: "MG_DIVERGED", 6: "MG_TIMEOUT"}

EXPORTED = [
    "mg_default_options", "mg_last_error", "mg_create", "mg_solve", "mg_get_solution_f64",
    "mg_level_shape", "mg_num_levels", "mg_apply_operator", "mg_smooth", "mg_residual_restrict",
    "mg_prolong_correct", "mg_precondition", "mg_destroy", "ns_create", "ns_step", "ns_momentum",
    "ns_divergence_rhs", "ns_correct", "ns_pressure_handle", "ns_destroy",
    "mg_profile_enable", "mg_profile_read", "mg_kernel_launches", "mg_vcycle_noalloc",
    "mg_create_batched", "mg_solve_batched", "mg_tune_batched", "mg_batched_config", "mg_destroy_batched",
    "gn_create", "gn_set_weights", "gn_get_weights", "gn_forward", "gn_gradients", "gn_adam_step",
    "gn_dataset_reserve", "gn_dataset_add", "gn_dataset_size", "gn_train", "gn_conv3d", "gn_conv3d_wgrad",
    "gn_destroy", "ns_set_guess", "ns_last_fields", "gn_kernel_launches", "ns_set_guess_level",
    "ns_coarse_fields", "ns_set_stencils", "ad_default_options", "ad_create", "ad_solve", "ad_num_levels",
    "ad_coarse_start", "ad_kernel_launches", "ad_destroy", "mg_probe_l2_read",
]
GN_NUM_WEIGHTS = 49680
GN_CONV_SCRATCH_BYTES = 28160
GN_WGRAD_SCRATCH_MIN = 256 + 27 * 16 * 16 * 4
GN_CONV_F32, GN_CONV_RELU, GN_CONV_DGRAD, GN_CONV_LIN = range(4)
GN_LOSS_L2, GN_LOSS_RESIDUAL = 0, 1
KERNEL_CLASSES = ["down_fine", "up_fine", "down", "up", "coarse", "p_update", "xr_update", "outer",
                  "init_finish", "momentum", "divergence", "correct", "cluster_pcg"]


class MgOptions(ctypes.Structure):
    _fields_ = [("pre", ctypes.c_int), ("post", ctypes.c_int), ("omega", ctypes.c_double),
                ("coarse_scale", ctypes.c_double), ("levels", ctypes.c_int), ("krylov", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("max_outer", ctypes.c_int), ("prec", ctypes.c_int),
                ("inner_floor", ctypes.c_double), ("cycle", ctypes.c_int), ("refine", ctypes.c_int)]


class MgStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer", ctypes.c_int),
                ("levels", ctypes.c_int), ("relres0", ctypes.c_double), ("relres", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("ms", ctypes.c_float), ("history", ctypes.c_double * 32),
                ("guess_relres", ctypes.c_double), ("guess_rejected", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "history"}
        d["history"] = [self.history[i] for i in range(min(self.outer + 1, 32))]
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_vp = ctypes.c_void_p
class AdOptions(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int), ("pre", ctypes.c_int), ("post", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_scale", ctypes.c_double), ("coarse_op", ctypes.c_int),
                ("levels", ctypes.c_int), ("max_cycles", ctypes.c_int)]


class AdStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int), ("relres0", ctypes.c_double),
                ("relres", ctypes.c_double), ("l1_first", ctypes.c_double), ("l1_last", ctypes.c_double),
                ("ms", ctypes.c_float)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_i64_3 = ctypes.c_int64 * 3
_d3 = ctypes.c_double * 3
_i6 = ctypes.c_int * 6


def load():
    """Load the library (built by ``paper_2402_17913_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libnpmg.so is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "mg_default_options": (None, [ctypes.POINTER(MgOptions)]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64_3, _d3, _i6, _vp,
                                     ctypes.POINTER(MgOptions), _vp]),
        "mg_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp, ctypes.POINTER(MgStats)]),
        "mg_get_solution_f64": (ctypes.c_int, [_vp, _vp, _vp]),
        "mg_level_shape": (ctypes.c_int, [_vp, ctypes.c_int, _i64_3]),
        "mg_num_levels": (ctypes.c_int, [_vp]),
        "mg_apply_operator": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
        "mg_smooth": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp]),
        "mg_residual_restrict": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]),
        "mg_prolong_correct": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
        "mg_precondition": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "mg_destroy": (ctypes.c_int, [_vp]),
        "ns_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64_3, ctypes.c_double, _vp,
                                     ctypes.c_double, ctypes.POINTER(MgOptions), _vp]),
        "ns_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, _vp, ctypes.POINTER(MgStats)]),
        "ns_momentum": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _vp]),
        "ns_divergence_rhs": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp]),
        "ns_correct": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, _vp]),
        "ns_pressure_handle": (_vp, [_vp]),
        "ns_destroy": (ctypes.c_int, [_vp]),
        "mg_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
        "mg_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.c_int]),
        "mg_kernel_launches": (ctypes.c_int64, [_vp]),
        "mg_vcycle_noalloc": (ctypes.c_int, [ctypes.c_int, _i64_3, _d3, _i6, _vp, ctypes.POINTER(MgOptions),
                                             _vp, _vp, _vp]),
        "mg_create_batched": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_int * 4,
                                             ctypes.POINTER(_vp), ctypes.POINTER(MgOptions), _vp]),
        "mg_solve_batched": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_double, _vp,
                                            ctypes.POINTER(MgStats)]),
        "mg_tune_batched": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_double, _vp,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
        "mg_batched_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int]),
        "mg_destroy_batched": (ctypes.c_int, [_vp]),
        "gn_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _vp]),
        "gn_set_weights": (ctypes.c_int, [_vp, _vp]),
        "gn_get_weights": (ctypes.c_int, [_vp, _vp]),
        "gn_forward": (ctypes.c_int, [_vp, ctypes.c_int, _i64_3, _vp, _vp, _vp, _vp]),
        "gn_gradients": (ctypes.c_int, [_vp, ctypes.c_int, _i64_3, _vp, _vp, _vp, _vp, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
        "gn_adam_step": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp]),
        "gn_dataset_reserve": (ctypes.c_int, [_vp, _i64_3, ctypes.c_int, ctypes.c_double]),
        "gn_dataset_add": (ctypes.c_int, [_vp, _i64_3, _vp, _vp, _vp, _vp, _vp]),
        "gn_dataset_size": (ctypes.c_int, [_vp]),
        "gn_train": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                    _vp, _vp]),
        "gn_conv3d": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _i64_3, ctypes.c_int, _vp, _vp]),
        "gn_conv3d_wgrad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _i64_3, _vp, ctypes.c_size_t, _vp]),
        "gn_destroy": (ctypes.c_int, [_vp]),
        "ns_set_guess": (ctypes.c_int, [_vp, _vp]),
        "ns_set_guess_level": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
        "ns_set_stencils": (ctypes.c_int, [_vp, ctypes.c_int]),
        "ad_default_options": (ctypes.c_int, [ctypes.POINTER(AdOptions)]),
        "ad_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64 * 2, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(AdOptions), _vp]),
        "ad_solve": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp,
                                    ctypes.POINTER(AdStats)]),
        "ad_num_levels": (ctypes.c_int, [_vp]),
        "ad_coarse_start": (ctypes.c_int, [_vp]),
        "ad_kernel_launches": (ctypes.c_int64, [_vp]),
        "ad_destroy": (ctypes.c_int, [_vp]),
        "ns_coarse_fields": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
        "gn_kernel_launches": (ctypes.c_int64, []),
        "ns_last_fields": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
        "mg_probe_l2_read": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int, _vp, ctypes.c_int, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error():
    return load().mg_last_error().decode()


def _check(status, allow=(MG_OK,)):
    if status not in allow:
        raise MGError(status, last_error())
    return status


def ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def default_options(**kw):
    o = MgOptions()
    load().mg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def mg_create(dim, shape, spacing, bc, solid=None, options=None, stream=None):
    """Returns an mg_handle (int).  shape/spacing in (x, y[, z]) order."""
    lib = load()
    h = _vp()
    shp = _i64_3(*(list(shape) + [1] * (3 - len(shape))))
    sp = _d3(*(list(spacing) + [1.0] * (3 - len(spacing))))
    b6 = _i6(*(list(bc) + [0] * (6 - len(bc))))
    opt = options if options is not None else default_options()
    _check(lib.mg_create(ctypes.byref(h), dim, shp, sp, b6, ptr(solid), ctypes.byref(opt), stream_ptr(stream)))
    return h.value


def mg_solve(h, b, x, rel_tol, stream=None, stats=True):
    """Solve in place into x; returns (status, stats dict or None)."""
    lib = load()
    st = MgStats() if stats else None
    status = lib.mg_solve(h, ptr(b), ptr(x), rel_tol, stream_ptr(stream), ctypes.byref(st) if stats else None)
    _check(status, allow=(MG_OK, MG_NOT_CONVERGED, MG_DIVERGED))
    return status, (st.as_dict() if stats else None)


def mg_get_solution_f64(h, x64, stream=None):
    _check(load().mg_get_solution_f64(h, ptr(x64), stream_ptr(stream)))


def mg_num_levels(h):
    return load().mg_num_levels(h)


def mg_level_shape(h, k):
    out = _i64_3()
    _check(load().mg_level_shape(h, k, out))
    return tuple(out)


def mg_apply_operator(h, k, x, y, stream=None):
    _check(load().mg_apply_operator(h, k, ptr(x), ptr(y), stream_ptr(stream)))


def mg_smooth(h, k, x, b, sweeps, stream=None):
    _check(load().mg_smooth(h, k, ptr(x), ptr(b), sweeps, stream_ptr(stream)))


def mg_residual_restrict(h, k, x, b, bc, stream=None):
    _check(load().mg_residual_restrict(h, k, ptr(x), ptr(b), ptr(bc), stream_ptr(stream)))


def mg_prolong_correct(h, k, e, x, stream=None):
    _check(load().mg_prolong_correct(h, k, ptr(e), ptr(x), stream_ptr(stream)))


def mg_precondition(h, r, z, stream=None):
    _check(load().mg_precondition(h, ptr(r), ptr(z), stream_ptr(stream)))


def mg_probe_l2_read(buf, reps, sink, stream=None):
    """One launch reading the float32 device tensor ``buf`` ``reps`` times
    (the L2 roof when ``buf`` fits in L2); ``sink`` holds one float per
    block (4 x the SM count)."""
    _check(load().mg_probe_l2_read(ptr(buf), buf.numel(), reps, ptr(sink), sink.numel(), stream_ptr(stream)))


def mg_destroy(h):
    if h:
        load().mg_destroy(h)


def ns_create(dim, cells, h, solid=None, sigma=1e8, options=None, stream=None):
    lib = load()
    out = _vp()
    c = _i64_3(*(list(cells) + [1] * (3 - len(cells))))
    opt = options if options is not None else default_options()
    _check(lib.ns_create(ctypes.byref(out), dim, c, h, ptr(solid), sigma, ctypes.byref(opt), stream_ptr(stream)))
    return out.value


def ns_step(ns, u, v, w, p, dt, nu, u_inflow, rel_tol, stream=None, stats=True):
    lib = load()
    st = MgStats() if stats else None
    status = lib.ns_step(ns, ptr(u), ptr(v), ptr(w), ptr(p), dt, nu, u_inflow, rel_tol, stream_ptr(stream),
                         ctypes.byref(st) if stats else None)
    _check(status, allow=(MG_OK, MG_NOT_CONVERGED, MG_DIVERGED))
    return status, (st.as_dict() if stats else None)


def ns_momentum(ns, u, v, w, p, us, vs, ws, dt, nu, u_inflow, stream=None):
    _check(load().ns_momentum(ns, ptr(u), ptr(v), ptr(w), ptr(p), ptr(us), ptr(vs), ptr(ws), dt, nu, u_inflow,
                              stream_ptr(stream)))


def ns_divergence_rhs(ns, us, vs, ws, dt, b, stream=None):
    _check(load().ns_divergence_rhs(ns, ptr(us), ptr(vs), ptr(ws), dt, ptr(b), stream_ptr(stream)))


def ns_correct(ns, u, v, w, p, dp, dt, stream=None):
    _check(load().ns_correct(ns, ptr(u), ptr(v), ptr(w), ptr(p), ptr(dp), dt, stream_ptr(stream)))


def ns_pressure_handle(ns):
    return load().ns_pressure_handle(ns)


def mg_profile_enable(h, on=True):
    _check(load().mg_profile_enable(h, 1 if on else 0))


def mg_profile_read(h, reset=True):
    """{class: (ms, launches)} accumulated since the last reset."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(load().mg_profile_read(h, ms, cnt, 1 if reset else 0))
    return {KERNEL_CLASSES[i]: (ms[i], cnt[i]) for i in range(n)}


def mg_kernel_launches(h):
    return load().mg_kernel_launches(h)


def mg_vcycle_noalloc(dim, shape, spacing, bc, r, z, solid=None, options=None, stream=None):
    """One preconditioner cycle z = M r without a handle or any device
    allocation (scratch in the library's static device array)."""
    shp = _i64_3(*(list(shape) + [1] * (3 - len(shape))))
    sp = _d3(*(list(spacing) + [1.0] * (3 - len(spacing))))
    b6 = _i6(*(list(bc) + [0] * (6 - len(bc))))
    opt = options if options is not None else default_options()
    return _check(load().mg_vcycle_noalloc(dim, shp, sp, b6, ptr(solid), ctypes.byref(opt), ptr(r), ptr(z),
                                           stream_ptr(stream)))


def _ptr_array(ts):
    return (_vp * len(ts))(*[ptr(t) for t in ts])


def mg_create_batched(shapes, spacings, bc, masks=None, options=None, stream=None):
    """shapes: list of (nx, ny); spacings: list of (hx, hy); masks: list of
    device uint8 tensors or None entries (or None)."""
    n = len(shapes)
    shp = (ctypes.c_int64 * (2 * n))(*[int(v) for s_ in shapes for v in s_])
    sp = (ctypes.c_double * (2 * n))(*[float(v) for s_ in spacings for v in s_])
    b4 = (ctypes.c_int * 4)(*bc)
    m = None if masks is None else _ptr_array(masks)
    opt = options if options is not None else default_options()
    out = _vp()
    _check(load().mg_create_batched(ctypes.byref(out), n, shp, sp, b4, m, ctypes.byref(opt), stream_ptr(stream)))
    return out.value


def mg_solve_batched(b, rhs, x, rel_tol, stream=None, stats=True):
    """rhs, x: lists of device tensors.  Returns (status, list of stats dicts)."""
    n = len(rhs)
    st = (MgStats * n)() if stats else None
    status = load().mg_solve_batched(b, _ptr_array(rhs), _ptr_array(x), rel_tol, stream_ptr(stream),
                                     st if stats else None)
    _check(status, allow=(MG_OK, MG_NOT_CONVERGED, MG_DIVERGED, MG_TIMEOUT))
    return status, ([s_.as_dict() for s_ in st] if stats else None)


def mg_tune_batched(b, rhs, x, rel_tol, stream=None):
    tx, ty, sw = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().mg_tune_batched(b, _ptr_array(rhs), _ptr_array(x), rel_tol, stream_ptr(stream), ctypes.byref(tx),
                                  ctypes.byref(ty), ctypes.byref(sw)))
    return tx.value, ty.value, sw.value


def mg_batched_config(b, tile_x, tile_y, sweeps, barrier_timeout_s=2.0, withhold_first_arrival=False):
    _check(load().mg_batched_config(b, tile_x, tile_y, sweeps, barrier_timeout_s, 1 if withhold_first_arrival else 0))


def mg_destroy_batched(b):
    if b:
        load().mg_destroy_batched(b)


def ns_destroy(ns):
    if ns:
        load().ns_destroy(ns)


# ---------------------------------------------------------------------------
# learned initial guess
def _host_f32(a, n=None):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    if n is not None and a.size != n:
        raise ValueError("expected %d floats, got %d" % (n, a.size))
    return a


def gn_flatten(weights):
    """Concatenate per-layer arrays [27][c_in][c_out] into the C layout."""
    import numpy as np
    return np.concatenate([np.asarray(w, dtype=np.float32).ravel() for w in weights])


def gn_unflatten(flat):
    """Inverse of gn_flatten (float64 arrays per layer)."""
    import numpy as np
    io = [(2, 16)] + [(16, 16)] * 7 + [(16, 1)]
    out, o = [], 0
    for ci, co in io:
        k = 27 * ci * co
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(27, ci, co))
        o += k
    return out


def gn_create(weights, stream=None):
    """weights: list of 9 arrays [27][c_in][c_out] or the flat C layout."""
    w = _host_f32(gn_flatten(weights) if isinstance(weights, (list, tuple)) else weights, GN_NUM_WEIGHTS)
    out = _vp()
    _check(load().gn_create(ctypes.byref(out), w.ctypes.data, stream_ptr(stream)))
    return out.value


def gn_set_weights(g, weights):
    w = _host_f32(gn_flatten(weights) if isinstance(weights, (list, tuple)) else weights, GN_NUM_WEIGHTS)
    _check(load().gn_set_weights(g, w.ctypes.data))


def gn_get_weights(g):
    import numpy as np
    w = np.empty(GN_NUM_WEIGHTS, np.float32)
    _check(load().gn_get_weights(g, w.ctypes.data))
    return w


def gn_forward(g, cells, b, p, out, n=1, stream=None):
    _check(load().gn_forward(g, n, _i64_3(*cells), ptr(b), ptr(p), ptr(out), stream_ptr(stream)))


def gn_gradients(g, cells, b, p, t=None, n=1, fluid=None, loss_mode=GN_LOSS_L2, h=1.0, stream=None):
    """Returns (loss, flat float32 gradient)."""
    import numpy as np
    loss = ctypes.c_double()
    grad = np.empty(GN_NUM_WEIGHTS, np.float32)
    _check(load().gn_gradients(g, n, _i64_3(*cells), ptr(b), ptr(p), ptr(t), ptr(fluid), loss_mode, h,
                               ctypes.byref(loss), grad.ctypes.data, stream_ptr(stream)))
    return loss.value, grad


def gn_adam_step(g, lr, grad=None, stream=None):
    gp = None if grad is None else _host_f32(grad, GN_NUM_WEIGHTS)
    _check(load().gn_adam_step(g, None if gp is None else gp.ctypes.data, lr, stream_ptr(stream)))


def gn_dataset_reserve(g, crop, capacity, h=1.0):
    _check(load().gn_dataset_reserve(g, _i64_3(*crop), capacity, h))


def gn_dataset_add(g, cells, b, p_next, dp, solid=None, stream=None):
    _check(load().gn_dataset_add(g, _i64_3(*cells), ptr(b), ptr(p_next), ptr(dp), ptr(solid), stream_ptr(stream)))


def gn_dataset_size(g):
    return load().gn_dataset_size(g)


def gn_train(g, steps, batch, seed, lr, loss_mode=GN_LOSS_RESIDUAL, stream=None):
    """Returns the per-step losses (numpy float64)."""
    import numpy as np
    losses = np.zeros(steps, np.float64)
    _check(load().gn_train(g, steps, batch, seed, lr, loss_mode, losses.ctypes.data, stream_ptr(stream)))
    return losses


def gn_conv3d(x, w, y, cells, n=1, mode=GN_CONV_F32, scratch=None, stream=None):
    """x: bf16 tensor [n][z][y][x][16]; w: float32 CUDA tensor [27][16][16]."""
    import torch
    if scratch is None:
        scratch = torch.empty(GN_CONV_SCRATCH_BYTES, dtype=torch.uint8, device=x.device)
    _check(load().gn_conv3d(ptr(x), ptr(w), ptr(y), n, _i64_3(*cells), mode, ptr(scratch), stream_ptr(stream)))


def gn_conv3d_wgrad(x, gr, dw, cells, n=1, scratch_bytes=None, stream=None):
    import torch
    nbytes = scratch_bytes or (GN_WGRAD_SCRATCH_MIN + 511 * 27 * 16 * 16 * 4)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    _check(load().gn_conv3d_wgrad(ptr(x), ptr(gr), ptr(dw), n, _i64_3(*cells), ptr(scratch), nbytes,
                                  stream_ptr(stream)))


def gn_kernel_launches():
    return load().gn_kernel_launches()


def gn_destroy(g):
    if g:
        load().gn_destroy(g)


def ns_set_guess(ns, g):
    _check(load().ns_set_guess(ns, g))


def ns_set_guess_level(ns, g, level):
    _check(load().ns_set_guess_level(ns, g, int(level)))


def ad_default_options(**kw):
    o = AdOptions()
    _check(load().ad_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ad_create(cells, h, dt, nu, u, v, scheme=AD_UPWIND, options=None, stream=None):
    """Implicit advection-diffusion step handle; cells = (nx, ny)."""
    out = _vp()
    opt = options if options is not None else ad_default_options()
    _check(load().ad_create(ctypes.byref(out), (ctypes.c_int64 * 2)(*cells), h, dt, nu, u, v, int(scheme),
                            ctypes.byref(opt), stream_ptr(stream)))
    return out.value


def ad_solve(hd, b, x, rel_tol=1e-6, l1_tol=0.0, x0=None, stream=None):
    """T^{n+1} into x from T^n = b (initial guess x0, default b); returns (status, stats)."""
    st = AdStats()
    status = load().ad_solve(hd, ptr(b), ptr(x0), ptr(x), rel_tol, l1_tol, stream_ptr(stream), ctypes.byref(st))
    _check(status, allow=(MG_OK, MG_NOT_CONVERGED, MG_DIVERGED))
    return status, st.as_dict()


def ad_num_levels(hd):
    return load().ad_num_levels(hd)


def ad_coarse_start(hd):
    return load().ad_coarse_start(hd)


def ad_kernel_launches(hd):
    return load().ad_kernel_launches(hd)


def ad_destroy(hd):
    if hd:
        load().ad_destroy(hd)


def ns_set_stencils(ns, stencil):
    """Momentum filters of later steps: NS_STENCIL_FD (5/7-point) or NS_STENCIL_FE (9/27-point)."""
    _check(load().ns_set_stencils(ns, int(stencil)))


def ns_coarse_fields(ns, level, p, b_c, p_c, dp_c, solid_c, stream=None):
    """Last step's b, dp and the given p restricted `level` times, solid coarsened."""
    _check(load().ns_coarse_fields(ns, int(level), ptr(p), ptr(b_c), ptr(p_c), ptr(dp_c), ptr(solid_c),
                                   stream_ptr(stream)))


def ns_last_fields(ns):
    """(b, dp) device pointers (ints) of the last ns_step."""
    b, dp = _vp(), _vp()
    _check(load().ns_last_fields(ns, ctypes.byref(b), ctypes.byref(dp)))
    return b.value, dp.value
