"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of the coupled step runs in the CUDA library.
Host arrays are numpy float64 / int32 in the layouts documented in lbm.h.
If the library has not been built the first call raises ``RuntimeError``;
there is no fallback path.

PyTorch is used only as plumbing: ``use_torch`` routes the library's device
allocations through the PyTorch caching allocator and runs its work on the
current PyTorch stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_ALLOC = -2
LBM_ERR_UNSTABLE = -3
LBM_ERR_TIMEOUT = -4
LBM_ERR_CUDA = -5
LBM_ERR_STATE = -6

LBM_WALL_XM, LBM_WALL_XP, LBM_WALL_YM, LBM_WALL_YP, LBM_WALL_ZM, LBM_WALL_ZP = (1 << k for k in range(6))
LBM_WALL_ALL = 0x3F
LBM_TOP_FREE_SLIP = 0x40
LBM_WALL_ALL_FREE_TOP = 0x7F

LBM_FORCE_LIFT = 0x1
LBM_FORCE_STRESS = 0x2
LBM_MAP_CELL = 0
LBM_MAP_POINT = 1
LBM_REACTION_DRAG_LIFT = 0
LBM_REACTION_ALL = 1

LBM_STORE_F32 = 0
LBM_STORE_F16 = 1
LBM_STORE_BF16 = 2
LBM_MAX_DIAMETER = 6.0


class LbmError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("%s: %s" % (_status_name(code), message))
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_double),
        ("rho_l", ctypes.c_double),
        ("rho_ratio", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("c_added_mass", ctypes.c_double),
        ("drag_scale", ctypes.c_double),
        ("sn_coeff", ctypes.c_double),
        ("sn_exp", ctypes.c_double),
        ("width_factor", ctypes.c_double),
        ("substeps", ctypes.c_int),
        ("two_way", ctypes.c_int),
        ("forces", ctypes.c_int),
        ("mapping", ctypes.c_int),
        ("reaction", ctypes.c_int),
    ]


class lbm_physical(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("dx", "dt", "rho_l", "rho_b", "mu_l", "sigma", "g", "rho_l_lu")]


class lbm_units(ctypes.Structure):
    _fields_ = [("lcf", ctypes.c_double), ("tcf", ctypes.c_double), ("mcf", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_lib = None


def lib():
    """Load liblbm.so (built by ``paper_1710_07073_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is not built (%s); run python -m paper_1710_07073_gb300.build"
                           % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, u, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_longlong
    P = ctypes.POINTER
    sig = {
        "lbm_default_params": (None, [P(lbm_params)]),
        "lbm_velocity_set": (None, [P(i), P(d)]),
        "lbm_units_from_physical": (i, [P(lbm_physical), P(lbm_units), P(lbm_params), P(d)]),
        "lbm_create": (i, [i, i, i, d, u, P(vp)]),
        "lbm_create_storage": (i, [i, i, i, d, u, i, d, P(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_set_stream": (i, [vp, vp]),
        "lbm_set_allocator": (i, [vp, ALLOC_FN, FREE_FN, vp]),
        "lbm_set_params": (i, [vp, P(lbm_params)]),
        "lbm_get_params": (i, [vp, P(lbm_params)]),
        "lbm_set_fields": (i, [vp, P(d), P(d)]),
        "lbm_set_populations": (i, [vp, P(d)]),
        "lbm_get_populations": (i, [vp, P(d)]),
        "lbm_set_bubbles": (i, [vp, i, P(d), P(d), P(d)]),
        "lbm_step": (i, [vp, i]),
        "lbm_get_fields": (i, [vp, P(d), P(d)]),
        "lbm_get_bubbles": (i, [vp, i, P(i), P(d), P(d), P(d), P(d), P(i)]),
        "lbm_get_totals": (i, [vp, P(d)]),
        "lbm_get_bins": (i, [vp, P(i), P(i), P(i), P(i), P(i), i, P(i)]),
        "lbm_sites": (ll, [vp]),
        "lbm_bytes_per_site": (i, [vp]),
        "lbm_set_kernel_timing": (i, [vp, i]),
        "lbm_get_kernel_time": (i, [vp, P(d), P(i)]),
        "lbm_launch_count": (ll, [vp]),
        "lbm_adj_forward": (i, [vp, i, i, i, d, P(d)]),
        "lbm_adj_backward": (i, [vp, d, P(d), P(d), P(d)]),
        "lbm_batch_create": (i, [i, P(i), P(d), P(u), i, d, P(vp)]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_set_stream": (i, [vp, vp]),
        "lbm_batch_set_allocator": (i, [vp, ALLOC_FN, FREE_FN, vp]),
        "lbm_batch_set_params": (i, [vp, P(lbm_params)]),
        "lbm_batch_set_bubbles": (i, [vp, P(i), P(d), P(d), P(d)]),
        "lbm_batch_step": (i, [vp, i]),
        "lbm_batch_tune": (i, [vp, i, P(i), P(i)]),
        "lbm_batch_launch_shape": (i, [vp, P(i), P(i), P(i)]),
        "lbm_batch_set_launch_shape": (i, [vp, i, i, i]),
        "lbm_batch_get_fields": (i, [vp, i, P(d), P(d)]),
        "lbm_batch_get_bubbles": (i, [vp, i, P(i), P(d), P(d), P(d), P(d), P(i)]),
        "lbm_batch_sites": (ll, [vp]),
        "lbm_batch_set_kernel_timing": (i, [vp, i]),
        "lbm_batch_get_kernel_time": (i, [vp, P(d), P(i)]),
        "lbm_batch_launch_count": (ll, [vp]),
        "lbm_batch_sync": (i, [vp]),
        "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
        "lbm_bin_bubbles_noalloc": (i, [i, i, i, u, i, vp, vp, vp, vp, vp, i, vp, vp]),
        "lbm_sweep_kernel": (ctypes.c_char_p, [vp]),
        "lbm_sync": (i, [vp]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_status_string": (ctypes.c_char_p, [i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _status_name(code):
    try:
        return lib().lbm_status_string(code).decode()
    except Exception:
        return str(code)


def _check(ctx, code):
    if code != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(code, msg)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


def _f64(a, size=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if size is not None and a.size != size:
        raise ValueError("expected %d values, got %d" % (size, a.size))
    return a


# ---- C entry points, same names ------------------------------------------------

def lbm_default_params():
    p = lbm_params()
    lib().lbm_default_params(ctypes.byref(p))
    return p


def lbm_velocity_set():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    lib().lbm_velocity_set(_iptr(c), _dptr(w))
    return c.reshape(19, 3), w


def lbm_units_from_physical(dx, dt, rho_l=1000.0, rho_b=1.0, mu_l=1e-3, sigma=0.073, g=9.81,
                            rho_l_lu=1.0, params=None):
    """Appendix A conversion (defaults: Table 3's water and air).  Returns
    (units, params, omega): units with lcf, tcf, mcf; ``params`` (a copy of
    the given lbm_params, else the defaults) with g, rho_l, rho_ratio and sigma
    in lattice units; omega from the lattice viscosity (Eq. 9)."""
    ph = lbm_physical(dx, dt, rho_l, rho_b, mu_l, sigma, g, rho_l_lu)
    u = lbm_units()
    p = lbm_default_params()
    if params is not None:
        ctypes.memmove(ctypes.byref(p), ctypes.byref(params), ctypes.sizeof(lbm_params))
    om = ctypes.c_double(0.0)
    rc = lib().lbm_units_from_physical(ctypes.byref(ph), ctypes.byref(u), ctypes.byref(p),
                                       ctypes.byref(om))
    if rc != LBM_OK:
        raise LbmError(rc, "physical set-up out of range")
    return u, p, om.value


def lbm_create(nx, ny, nz, omega, walls=LBM_WALL_ALL):
    h = ctypes.c_void_p()
    _check(None, lib().lbm_create(nx, ny, nz, float(omega), walls, ctypes.byref(h)))
    return h


def lbm_create_storage(nx, ny, nz, omega, walls, storage, scale=1.0):
    h = ctypes.c_void_p()
    _check(None, lib().lbm_create_storage(nx, ny, nz, float(omega), walls, storage, float(scale),
                                          ctypes.byref(h)))
    return h


def lbm_destroy(ctx):
    lib().lbm_destroy(ctx)


def lbm_set_stream(ctx, stream_handle):
    _check(ctx, lib().lbm_set_stream(ctx, ctypes.c_void_p(stream_handle)))


def lbm_set_allocator(ctx, alloc, free, user=None):
    _check(ctx, lib().lbm_set_allocator(ctx, alloc, free, user))


def lbm_set_params(ctx, params):
    _check(ctx, lib().lbm_set_params(ctx, ctypes.byref(params)))


def lbm_get_params(ctx):
    p = lbm_params()
    _check(ctx, lib().lbm_get_params(ctx, ctypes.byref(p)))
    return p


def lbm_sites(ctx):
    return int(lib().lbm_sites(ctx))


def lbm_bytes_per_site(ctx):
    return int(lib().lbm_bytes_per_site(ctx))


def lbm_set_fields(ctx, rho=None, u3=None):
    S = lbm_sites(ctx)
    r = _f64(rho, S)
    u = _f64(u3, 3 * S)
    _check(ctx, lib().lbm_set_fields(ctx, _dptr(r), _dptr(u)))


def lbm_set_populations(ctx, f):
    f = _f64(f, 19 * lbm_sites(ctx))
    _check(ctx, lib().lbm_set_populations(ctx, _dptr(f)))


def lbm_get_populations(ctx):
    out = np.empty(19 * lbm_sites(ctx), dtype=np.float64)
    _check(ctx, lib().lbm_get_populations(ctx, _dptr(out)))
    return out


def lbm_set_bubbles(ctx, pos3, vel3, diam):
    d = _f64(diam).reshape(-1)
    n = d.size
    p = _f64(pos3, 3 * n)
    v = _f64(vel3, 3 * n) if vel3 is not None else None
    _check(ctx, lib().lbm_set_bubbles(ctx, n, _dptr(p), _dptr(v), _dptr(d)))


def lbm_step(ctx, nsteps=1):
    _check(ctx, lib().lbm_step(ctx, int(nsteps)))


def lbm_get_fields(ctx, rho=True, u=True, out_rho=None, out_u=None):
    """Returns (rho[S], u[3S]); ``out_rho`` / ``out_u`` may supply float64 buffers
    (e.g. pinned host memory) to fill instead of new arrays."""
    S = lbm_sites(ctx)
    r = out_rho if out_rho is not None else (np.empty(S, dtype=np.float64) if rho else None)
    v = out_u if out_u is not None else (np.empty(3 * S, dtype=np.float64) if u else None)
    for a, size in ((r, S), (v, 3 * S)):
        if a is not None and (a.dtype != np.float64 or a.size != size or not a.flags.c_contiguous):
            raise ValueError("output buffer must be contiguous float64 of %d values" % size)
    _check(ctx, lib().lbm_get_fields(ctx, _dptr(r), _dptr(v)))
    return r, v


def lbm_get_bubbles(ctx, cap=None):
    n = ctypes.c_int(0)
    _check(ctx, lib().lbm_get_bubbles(ctx, 0, ctypes.byref(n), None, None, None, None, None))
    k = n.value if cap is None else min(cap, n.value)
    pos = np.empty(3 * k)
    vel = np.empty(3 * k)
    ul = np.empty(3 * k)
    psi = np.empty(3 * k)
    act = np.empty(k, dtype=np.int32)
    if k:
        _check(ctx, lib().lbm_get_bubbles(ctx, k, ctypes.byref(n), _dptr(pos), _dptr(vel),
                                          _dptr(ul), _dptr(psi), _iptr(act)))
    return {"pos": pos.reshape(k, 3), "vel": vel.reshape(k, 3), "ul": ul.reshape(k, 3),
            "psi": psi.reshape(k, 3), "active": act.astype(bool)}


def lbm_get_totals(ctx):
    out = np.empty(4)
    _check(ctx, lib().lbm_get_totals(ctx, _dptr(out)))
    return out


def lbm_get_bins(ctx):
    n = ctypes.c_int(0)
    _check(ctx, lib().lbm_get_bubbles(ctx, 0, ctypes.byref(n), None, None, None, None, None))
    tile = np.zeros(3, dtype=np.int32)
    nt = ctypes.c_int(0)
    nitems = ctypes.c_int(0)
    _check(ctx, lib().lbm_get_bins(ctx, None, _iptr(tile), ctypes.byref(nt), None, None, 0,
                                   ctypes.byref(nitems)))
    cell = np.empty(n.value, dtype=np.int32)
    off = np.empty(nt.value + 1, dtype=np.int32)
    items = np.empty(max(nitems.value, 1), dtype=np.int32)
    _check(ctx, lib().lbm_get_bins(ctx, _iptr(cell), _iptr(tile), ctypes.byref(nt), _iptr(off),
                                   _iptr(items), items.size, ctypes.byref(nitems)))
    return {"cell": cell, "tile": tuple(int(t) for t in tile), "offsets": off,
            "items": items[:nitems.value]}


def lbm_set_kernel_timing(ctx, on=True):
    _check(ctx, lib().lbm_set_kernel_timing(ctx, 1 if on else 0))


def lbm_get_kernel_time(ctx):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _check(ctx, lib().lbm_get_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lbm_adj_forward(ctx, nsteps, checkpoint_every, window, target):
    """Forward record of nsteps steps; returns L = (ubar - target)^2."""
    loss = ctypes.c_double(0.0)
    _check(ctx, lib().lbm_adj_forward(ctx, int(nsteps), int(checkpoint_every), int(window),
                                      float(target), ctypes.byref(loss)))
    return loss.value


def lbm_adj_backward(ctx, dloss=1.0, want_u0=True):
    """Adjoint sweep: (dL/ds_D, dL/dd_b[n], dL/du0[3S] or None), scaled by dloss."""
    n = ctypes.c_int(0)
    _check(ctx, lib().lbm_get_bubbles(ctx, 0, ctypes.byref(n), None, None, None, None, None))
    g_sd = ctypes.c_double(0.0)
    g_d = np.zeros(n.value)
    g_u0 = np.zeros(3 * lbm_sites(ctx)) if want_u0 else None
    _check(ctx, lib().lbm_adj_backward(ctx, float(dloss), ctypes.byref(g_sd), _dptr(g_d),
                                       _dptr(g_u0)))
    return g_sd.value, g_d, g_u0


LBM_NOALLOC_MAX_TILES = 262144
LBM_NOALLOC_MAX_HALF_WIDTH = 9.0
LBM_NOALLOC_STATUS_OVERFLOW = 1
LBM_NOALLOC_STATUS_SKIPPED = 2


def lbm_bin_bubbles_noalloc(nx, ny, nz, walls, n, pos3_ptr, half_width_ptr, active_ptr,
                            tile_offsets_ptr, tile_items_ptr, cap_items, status_ptr, stream=0):
    """Bin bubbles into tiles without any allocation in the library.

    Every pointer is a device address (an int, e.g. ``tensor.data_ptr()``) of
    caller-owned memory; see lbm.h.  Raises LbmError on a bad argument."""
    code = lib().lbm_bin_bubbles_noalloc(nx, ny, nz, walls, n, pos3_ptr, half_width_ptr,
                                         active_ptr, tile_offsets_ptr, tile_items_ptr,
                                         int(cap_items), status_ptr, stream)
    if code != LBM_OK:
        raise LbmError(code, "lbm_bin_bubbles_noalloc")


def lbm_launch_count(ctx):
    return int(lib().lbm_launch_count(ctx))


def lbm_sweep_kernel(ctx):
    return lib().lbm_sweep_kernel(ctx).decode()


def lbm_sync(ctx):
    _check(ctx, lib().lbm_sync(ctx))


def lbm_last_error(ctx):
    return lib().lbm_last_error(ctx).decode()


def lbm_status_string(code):
    return lib().lbm_status_string(code).decode()


# ---- batches ---------------------------------------------------------------------

def _bcheck(b, code):
    if code != LBM_OK:
        raise LbmError(code, lib().lbm_batch_last_error(b).decode() if b else "")


def lbm_batch_create(dims_list, omegas, walls=None, storage=LBM_STORE_F32, scale=1.0):
    n = len(dims_list)
    dims = np.ascontiguousarray(np.asarray(dims_list, dtype=np.int32).reshape(-1))
    om = _f64(omegas, n)
    w = None
    if walls is not None:
        w = np.ascontiguousarray(np.asarray(walls, dtype=np.uint32))
    h = ctypes.c_void_p()
    code = lib().lbm_batch_create(n, _iptr(dims), _dptr(om),
                                  w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)) if w is not None
                                  else None, storage, float(scale), ctypes.byref(h))
    _bcheck(None, code)
    return h


def lbm_batch_destroy(b):
    lib().lbm_batch_destroy(b)


def lbm_batch_set_stream(b, stream_handle):
    _bcheck(b, lib().lbm_batch_set_stream(b, ctypes.c_void_p(stream_handle)))


def lbm_batch_set_allocator(b, alloc, free, user=None):
    _bcheck(b, lib().lbm_batch_set_allocator(b, alloc, free, user))


def lbm_batch_set_params(b, params):
    _bcheck(b, lib().lbm_batch_set_params(b, ctypes.byref(params)))


def lbm_batch_set_bubbles(b, counts, pos3, vel3, diam):
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    d = _f64(diam).reshape(-1)
    p = _f64(pos3, 3 * d.size)
    v = _f64(vel3, 3 * d.size) if vel3 is not None else None
    _bcheck(b, lib().lbm_batch_set_bubbles(b, _iptr(c), _dptr(p), _dptr(v), _dptr(d)))


def lbm_batch_step(b, nsteps=1):
    _bcheck(b, lib().lbm_batch_step(b, int(nsteps)))


def lbm_batch_tune(b, trial_steps=10):
    depth = ctypes.c_int(0)
    grid = ctypes.c_int(0)
    _bcheck(b, lib().lbm_batch_tune(b, int(trial_steps), ctypes.byref(depth), ctypes.byref(grid)))
    return depth.value, grid.value


def lbm_batch_set_launch_shape(b, planes, depth, grid=0):
    _bcheck(b, lib().lbm_batch_set_launch_shape(b, int(planes), int(depth), int(grid)))


def lbm_batch_launch_shape(b):
    """(planes per CTA, z-blocks per work item, persistent CTAs)."""
    planes, depth, grid = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _bcheck(b, lib().lbm_batch_launch_shape(b, ctypes.byref(planes), ctypes.byref(depth),
                                            ctypes.byref(grid)))
    return planes.value, depth.value, grid.value


def lbm_batch_get_fields(b, col, sites, rho=True, u=True, out_rho=None, out_u=None):
    """Fields of column ``col`` (``sites`` nodes); ``out_rho`` / ``out_u`` may
    supply float64 buffers (e.g. pinned host memory) to fill."""
    r = out_rho if out_rho is not None else (np.empty(sites, dtype=np.float64) if rho else None)
    v = out_u if out_u is not None else (np.empty(3 * sites, dtype=np.float64) if u else None)
    for a, size in ((r, sites), (v, 3 * sites)):
        if a is not None and (a.dtype != np.float64 or a.size != size or not a.flags.c_contiguous):
            raise ValueError("output buffer must be contiguous float64 of %d values" % size)
    _bcheck(b, lib().lbm_batch_get_fields(b, int(col), _dptr(r), _dptr(v)))
    return r, v


def lbm_batch_get_bubbles(b):
    n = ctypes.c_int(0)
    _bcheck(b, lib().lbm_batch_get_bubbles(b, 0, ctypes.byref(n), None, None, None, None, None))
    k = n.value
    pos, vel, ul, psi = (np.empty(3 * k) for _ in range(4))
    act = np.empty(k, dtype=np.int32)
    if k:
        _bcheck(b, lib().lbm_batch_get_bubbles(b, k, ctypes.byref(n), _dptr(pos), _dptr(vel),
                                               _dptr(ul), _dptr(psi), _iptr(act)))
    return {"pos": pos.reshape(k, 3), "vel": vel.reshape(k, 3), "ul": ul.reshape(k, 3),
            "psi": psi.reshape(k, 3), "active": act.astype(bool)}


def lbm_batch_sites(b):
    return int(lib().lbm_batch_sites(b))


def lbm_batch_set_kernel_timing(b, on=True):
    _bcheck(b, lib().lbm_batch_set_kernel_timing(b, 1 if on else 0))


def lbm_batch_get_kernel_time(b):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _bcheck(b, lib().lbm_batch_get_kernel_time(b, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lbm_batch_launch_count(b):
    return int(lib().lbm_batch_launch_count(b))


def lbm_batch_sync(b):
    _bcheck(b, lib().lbm_batch_sync(b))


def lbm_batch_last_error(b):
    return lib().lbm_batch_last_error(b).decode()


class Batch:
    """Owning wrapper of a batch of independent columns."""

    def __init__(self, dims_list, omegas, walls=None, storage=LBM_STORE_F32, scale=1.0,
                 params=None):
        self.dims = [tuple(int(v) for v in d) for d in dims_list]
        self.h = lbm_batch_create(self.dims, omegas, walls, storage, scale)
        if params is not None:
            lbm_batch_set_params(self.h, params)

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fields(self, col):
        nx, ny, nz = self.dims[col]
        rho, u = lbm_batch_get_fields(self.h, col, nx * ny * nz)
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)


# ---- PyTorch plumbing ------------------------------------------------------------

_keepalive = {}


def use_torch(ctx, device=None):
    """Allocate the context's device memory from the PyTorch caching allocator and
    run its work on PyTorch's current stream of ``device``."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)

    def _alloc(nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev.index)
        except Exception:
            return None

    def _free(ptr, _nbytes, _user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _keepalive[ctx.value] = (a, f)
    lbm_set_allocator(ctx, a, f)
    lbm_set_stream(ctx, torch.cuda.current_stream(dev).cuda_stream)


class Column:
    """Owning wrapper of one context (destroys it when collected)."""

    def __init__(self, dims, omega, walls=LBM_WALL_ALL, storage=LBM_STORE_F32, scale=1.0,
                 params=None, torch_plumbing=False):
        nx, ny, nz = (int(v) for v in dims)
        self.dims = (nx, ny, nz)
        self.omega = float(omega)
        self.walls = int(walls)
        if storage == LBM_STORE_F32:
            self.ctx = lbm_create(nx, ny, nz, omega, walls)
        else:
            self.ctx = lbm_create_storage(nx, ny, nz, omega, walls, storage, scale)
        if torch_plumbing:
            use_torch(self.ctx)
        if params is not None:
            lbm_set_params(self.ctx, params)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_destroy(self.ctx)
            _keepalive.pop(self.ctx.value, None)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # Convenience accessors in [z, y, x] array order.
    def fields(self):
        nx, ny, nz = self.dims
        rho, u = lbm_get_fields(self.ctx)
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)
