"""Thin ctypes binding of libsidp (argument marshalling only).

Every function here has the name of the C entry point it calls (``include/sidp.h``) and only
converts arguments: numpy float64 arrays in and out, status codes to exceptions.  All
computation happens in the library's CUDA kernels.  ``Solver`` bundles the calls for one
context.  The library must have been built (``paper_2004_08503_gb300.build``); loading fails
loudly otherwise.
"""
import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsidp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sidp.h")

LAWS = {"burgers": 1, "euler": 2, "advection": 3, "advection_var": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}
BCS = {"periodic": 0, "outflow": 1, "exact": 2, "wall": 3, "split": 4}
LIMITERS = {"none": 0, "lo": 1, "subcell": 2, "elementwise": 3}
SIDES = {"W": 0, "E": 1, "S": 2, "N": 3}


class sidp_config(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int), ("p", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("precision", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("cfl", ctypes.c_double), ("gamma", ctypes.c_double), ("adv_beta", ctypes.c_double * 2),
                ("limiter", ctypes.c_int), ("smoothness", ctypes.c_int), ("si_s0", ctypes.c_double),
                ("si_kappa", ctypes.c_double), ("si_gmin", ctypes.c_double), ("si_gmax", ctypes.c_double),
                ("adv_grad", ctypes.c_double * 2), ("unsparsified", ctypes.c_int)]


class sidp_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_longlong), ("last_dt", ctypes.c_double),
                ("mass", ctypes.c_double * 4), ("umin", ctypes.c_double * 4), ("umax", ctypes.c_double * 4),
                ("rho_min", ctypes.c_double), ("p_min", ctypes.c_double),
                ("max_bound_violation", ctypes.c_double), ("max_entropy_violation", ctypes.c_double),
                ("rootfind_max_iters", ctypes.c_int), ("rootfind_cap_hits", ctypes.c_longlong),
                ("nonfinite", ctypes.c_longlong), ("bound_nudges", ctypes.c_longlong)]


class SidpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsidp status {status}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "sidp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(sidp_config), _P]),
    "sidp_destroy": (ctypes.c_int, [_P]),
    "sidp_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]),
    "sidp_node_coords": (ctypes.c_int, [_P, _D, _D]),
    "sidp_set_state": (ctypes.c_int, [_P, _D]),
    "sidp_get_state": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "sidp_set_ghost_state": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "sidp_set_split_boundary": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]),
    "sidp_set_time": (ctypes.c_int, [_P, ctypes.c_double]),
    "sidp_curved_metrics": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           _D, _D, _D]),
    "sidp_set_geometry": (ctypes.c_int, [_P, _D, _D]),
    "sidp_upload_state": (ctypes.c_int, [_P, _P]),
    "sidp_download_state": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "sidp_device_state": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    "sidp_compute_dt": (ctypes.c_int, [_P, _D]),
    "sidp_compute_dt_static": (ctypes.c_int, [ctypes.POINTER(sidp_config), _P, _P, _P]),
    "sidp_stage": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "sidp_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_set_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sidp_get_tile_index": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "sidp_set_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_set_stats": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_set_debug": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_get_bounds": (ctypes.c_int, [_P, _D, _D, _D, _D]),
    "sidp_get_diag": (ctypes.c_int, [_P, ctypes.POINTER(sidp_diag)]),
    "sidp_synchronize": (ctypes.c_int, [_P]),
    "sidp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sidp_last_error": (ctypes.c_char_p, [_P]),
    "sidp_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(sidp_config), ctypes.c_int, _P]),
    "sidp_batch_destroy": (ctypes.c_int, [_P]),
    "sidp_batch_sizes": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]),
    "sidp_batch_total_nodes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "sidp_batch_node_coords": (ctypes.c_int, [_P, ctypes.c_int, _D, _D]),
    "sidp_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "sidp_batch_set_geometry": (ctypes.c_int, [_P, ctypes.c_int, _D, _D]),
    "sidp_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "sidp_batch_get_buffer": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
    "sidp_fma_peak": (ctypes.c_int, [ctypes.c_int, _D, _P]),
    "sidp_batch_stage": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "sidp_batch_set_debug": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_batch_get_bounds": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D, _D]),
    "sidp_batch_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_batch_get_diag": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(sidp_diag)]),
    "sidp_batch_synchronize": (ctypes.c_int, [_P]),
    "sidp_batch_set_stats": (ctypes.c_int, [_P, ctypes.c_int]),
    "sidp_batch_last_error": (ctypes.c_char_p, [_P]),
}


def load():
    """Load libsidp.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_2004_08503_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


def header_functions():
    """Names of the entry points declared in include/sidp.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(sidp_\w+)\s*\(", txt)))


def _ptr(a):
    return a.ctypes.data_as(_D)


def _check(st, handle=None, err_fn="sidp_last_error"):
    if st != 0:
        lib = load()
        msg = getattr(lib, err_fn)(handle)
        raise SidpError(st, (lib.sidp_status_str(st) or b"").decode() + ": " + (msg or b"").decode())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def make_config(law="euler", p=3, nx=8, ny=8, precision="fp64", domain=(0.0, 1.0, 0.0, 1.0),
                bc=("periodic",) * 4, cfl=0.5, gamma=1.4, beta=(1.0, 0.0), limiter="subcell", smoothness=None,
                grad=(0.0, 0.0), sparsify=True):
    """smoothness: None, or dict(gmin, gmax[, s0, kappa]) for the Sec. 4.4 indicator.
    law "advection_var": velocity (beta[0] + grad[0] y, beta[1] + grad[1] x).
    sparsify=False: the unsparsified graph-viscosity comparison mode (Sec. 3.4)."""
    c = sidp_config()
    c.law, c.p, c.nx, c.ny = LAWS[law], p, nx, ny
    c.precision = PRECISIONS[precision]
    c.x0, c.x1, c.y0, c.y1 = domain
    for i, b in enumerate(bc):
        c.bc[i] = BCS[b]
    c.cfl, c.gamma = cfl, gamma
    c.adv_beta[0], c.adv_beta[1] = beta
    c.adv_grad[0], c.adv_grad[1] = grad
    c.unsparsified = 0 if sparsify else 1
    c.limiter = LIMITERS[limiter]
    if smoothness is not None:
        c.smoothness = 1
        c.si_gmin, c.si_gmax = smoothness["gmin"], smoothness["gmax"]
        c.si_s0 = smoothness.get("s0", 0.0)
        c.si_kappa = smoothness.get("kappa", 0.0)
    return c


# ------------------------------------------------------------------ same-name wrappers
def sidp_create(cfg, stream=None):
    h = _P()
    _check(load().sidp_create(ctypes.byref(h), ctypes.byref(cfg), _stream_handle(stream)))
    return h


def sidp_destroy(ctx):
    _check(load().sidp_destroy(ctx))


def sidp_sizes(ctx):
    n, nc = ctypes.c_longlong(), ctypes.c_int()
    _check(load().sidp_sizes(ctx, ctypes.byref(n), ctypes.byref(nc)), ctx)
    return n.value, nc.value


def sidp_node_coords(ctx):
    n, _ = sidp_sizes(ctx)
    x, y = np.empty(n), np.empty(n)
    _check(load().sidp_node_coords(ctx, _ptr(x), _ptr(y)), ctx)
    return x, y


def sidp_set_state(ctx, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(load().sidp_set_state(ctx, _ptr(u)), ctx)


def sidp_get_state(ctx, which=0):
    n, nc = sidp_sizes(ctx)
    u = np.empty((nc, n))
    _check(load().sidp_get_state(ctx, which, _ptr(u)), ctx)
    return u


def sidp_upload_state(ctx, host_ptr):
    """host_ptr: address of a host buffer in the storage type (e.g. a pinned torch tensor's data_ptr())."""
    _check(load().sidp_upload_state(ctx, host_ptr), ctx)


def sidp_download_state(ctx, which, host_ptr):
    _check(load().sidp_download_state(ctx, which, host_ptr), ctx)


def sidp_set_ghost_state(ctx, side, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(load().sidp_set_ghost_state(ctx, SIDES.get(side, side), _ptr(u)), ctx)


SIDES = {"W": 0, "E": 1, "S": 2, "N": 3}


def sidp_set_split_boundary(ctx, side, s0, speed, state_a, state_b=None):
    """side: 0..3 or "W", "E", "S", "N"; state_b None: a slip wall on that part."""
    side = SIDES.get(side, side)
    a = np.ascontiguousarray(state_a, dtype=np.float64)
    b = None if state_b is None else np.ascontiguousarray(state_b, dtype=np.float64)
    _check(load().sidp_set_split_boundary(ctx, int(side), ctypes.c_double(s0), ctypes.c_double(speed), _ptr(a),
                                          _ptr(b) if b is not None else None), ctx)


def sidp_set_time(ctx, t):
    _check(load().sidp_set_time(ctx, ctypes.c_double(t)), ctx)


GEO_FIELDS = 13


def sidp_curved_metrics(p, nx, ny, bc, x, y):
    """Metric arrays (GEO_FIELDS, N) of the curved mesh with node coordinates x, y (host only)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    out = np.empty((GEO_FIELDS, x.size))
    b = (ctypes.c_int * 4)(*[BCS.get(v, v) for v in bc])
    _check(load().sidp_curved_metrics(int(p), int(nx), int(ny), b, _ptr(x), _ptr(y), _ptr(out)))
    return out


def sidp_set_geometry(ctx, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    _check(load().sidp_set_geometry(ctx, _ptr(x), _ptr(y)), ctx)


def sidp_device_state(ctx):
    p, dt, st = _P(), ctypes.c_int(), ctypes.c_longlong()
    _check(load().sidp_device_state(ctx, ctypes.byref(p), ctypes.byref(dt), ctypes.byref(st)), ctx)
    return p.value, dt.value, st.value


def sidp_compute_dt(ctx):
    d = ctypes.c_double()
    _check(load().sidp_compute_dt(ctx, ctypes.byref(d)), ctx)
    return d.value


def sidp_compute_dt_static(cfg, d_state, d_dt, stream=None):
    """Time step for a caller-owned device state (device pointers as ints); allocates nothing."""
    _check(load().sidp_compute_dt_static(ctypes.byref(cfg), d_state, d_dt, _stream_handle(stream)))


def sidp_stage(ctx, k, dt):
    _check(load().sidp_stage(ctx, k, dt), ctx)


def sidp_step(ctx, nsteps=1):
    _check(load().sidp_step(ctx, nsteps), ctx)


def sidp_get_tile(ctx):
    tx, ty = ctypes.c_int(), ctypes.c_int()
    _check(load().sidp_get_tile(ctx, ctypes.byref(tx), ctypes.byref(ty)), ctx)
    return tx.value, ty.value


def sidp_get_tile_index(ctx):
    i = ctypes.c_int()
    _check(load().sidp_get_tile_index(ctx, ctypes.byref(i)), ctx)
    return i.value


def sidp_set_tile(ctx, index):
    _check(load().sidp_set_tile(ctx, int(index)), ctx)


def sidp_set_graph(ctx, on):
    _check(load().sidp_set_graph(ctx, int(on)), ctx)


def sidp_set_stats(ctx, on):
    _check(load().sidp_set_stats(ctx, int(on)), ctx)


def sidp_set_debug(ctx, on):
    _check(load().sidp_set_debug(ctx, int(on)), ctx)


def sidp_get_bounds(ctx):
    n, _ = sidp_sizes(ctx)
    out = [np.empty(n) for _ in range(4)]
    _check(load().sidp_get_bounds(ctx, *[_ptr(o) for o in out]), ctx)
    return dict(zip(("lo", "hi", "K", "alpha"), out))


def _diag_dict(d):
    return {f: (list(getattr(d, f)) if isinstance(getattr(d, f), ctypes.Array) else getattr(d, f))
            for f, _ in sidp_diag._fields_}


def sidp_get_diag(ctx):
    d = sidp_diag()
    _check(load().sidp_get_diag(ctx, ctypes.byref(d)), ctx)
    return _diag_dict(d)


def sidp_synchronize(ctx):
    _check(load().sidp_synchronize(ctx), ctx)


def sidp_status_str(st):
    return load().sidp_status_str(st).decode()


def sidp_batch_create(cfgs, stream=None):
    arr = (sidp_config * len(cfgs))(*cfgs)
    h = _P()
    st = load().sidp_batch_create(ctypes.byref(h), arr, len(cfgs), _stream_handle(stream))
    _check(st, None, "sidp_batch_last_error")
    return h


def _bcheck(st, b):
    _check(st, b, "sidp_batch_last_error")


def sidp_batch_destroy(b):
    _bcheck(load().sidp_batch_destroy(b), b)


def sidp_batch_sizes(b, i):
    n, nc = ctypes.c_longlong(), ctypes.c_int()
    _bcheck(load().sidp_batch_sizes(b, i, ctypes.byref(n), ctypes.byref(nc)), b)
    return n.value, nc.value


def sidp_batch_total_nodes(b):
    n = ctypes.c_longlong()
    _bcheck(load().sidp_batch_total_nodes(b, ctypes.byref(n)), b)
    return n.value


def sidp_batch_node_coords(b, i):
    n, _ = sidp_batch_sizes(b, i)
    x, y = np.empty(n), np.empty(n)
    _bcheck(load().sidp_batch_node_coords(b, i, _ptr(x), _ptr(y)), b)
    return x, y


def sidp_batch_set_geometry(b, i, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    n, _ = sidp_batch_sizes(b, i)
    if x.size != n or y.size != n:
        raise ValueError(f"instance {i} has {n} nodes; got {x.size} and {y.size} coordinates")
    _bcheck(load().sidp_batch_set_geometry(b, i, _ptr(x), _ptr(y)), b)


def sidp_batch_set_state(b, i, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    _bcheck(load().sidp_batch_set_state(b, i, _ptr(u)), b)


def sidp_batch_get_state(b, i):
    n, nc = sidp_batch_sizes(b, i)
    u = np.empty((nc, n))
    _bcheck(load().sidp_batch_get_state(b, i, _ptr(u)), b)
    return u


def sidp_batch_get_buffer(b, i, which):
    n, nc = sidp_batch_sizes(b, i)
    u = np.empty((nc, n))
    _bcheck(load().sidp_batch_get_buffer(b, i, which, _ptr(u)), b)
    return u


def sidp_batch_stage(b, k, dt):
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    _bcheck(load().sidp_batch_stage(b, k, _ptr(dt)), b)


def sidp_batch_set_debug(b, on):
    _bcheck(load().sidp_batch_set_debug(b, int(on)), b)


def sidp_batch_get_bounds(b, i):
    n, _ = sidp_batch_sizes(b, i)
    out = [np.empty(n) for _ in range(4)]
    _bcheck(load().sidp_batch_get_bounds(b, i, *[_ptr(o) for o in out]), b)
    return dict(zip(("lo", "hi", "K", "alpha"), out))


def sidp_fma_peak(precision, stream=None):
    """Measured FMA throughput in flop/s ("mixed": float32, "fp64": float64)."""
    out = ctypes.c_double()
    _check(load().sidp_fma_peak(PRECISIONS[precision], ctypes.byref(out), _stream_handle(stream)))
    return out.value


def sidp_batch_step(b, nsteps=1):
    _bcheck(load().sidp_batch_step(b, nsteps), b)


def sidp_batch_get_diag(b, i):
    d = sidp_diag()
    _bcheck(load().sidp_batch_get_diag(b, i, ctypes.byref(d)), b)
    return _diag_dict(d)


def sidp_batch_set_stats(b, on):
    _bcheck(load().sidp_batch_set_stats(b, int(on)), b)


def sidp_batch_synchronize(b):
    _bcheck(load().sidp_batch_synchronize(b), b)


class Solver:
    """One problem instance (a libsidp context)."""

    def __init__(self, stream=None, **cfg):
        self.cfg = make_config(**cfg)
        self.ctx = sidp_create(self.cfg, stream)
        self.N, self.nc = sidp_sizes(self.ctx)

    def close(self):
        if self.ctx:
            sidp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def node_coords(self):
        return sidp_node_coords(self.ctx)

    def set_state(self, u):
        sidp_set_state(self.ctx, np.asarray(u).reshape(self.nc, self.N))

    def get_state(self, which=0):
        return sidp_get_state(self.ctx, which)

    def set_ghost(self, side, u):
        sidp_set_ghost_state(self.ctx, side, u)

    def set_split(self, side, s0, speed, a, b=None):
        sidp_set_split_boundary(self.ctx, side, s0, speed, a, b)

    def set_time(self, t):
        sidp_set_time(self.ctx, t)

    def set_geometry(self, x, y):
        """Curved mesh: node coordinates in library order (see sidp_set_geometry)."""
        sidp_set_geometry(self.ctx, x, y)

    def compute_dt(self):
        return sidp_compute_dt(self.ctx)

    def stage(self, k, dt):
        sidp_stage(self.ctx, k, dt)

    def step(self, n=1):
        sidp_step(self.ctx, n)

    def diag(self):
        return sidp_get_diag(self.ctx)

    def bounds(self):
        return sidp_get_bounds(self.ctx)

    def set_debug(self, on):
        sidp_set_debug(self.ctx, on)

    def set_stats(self, on):
        sidp_set_stats(self.ctx, on)

    def set_graph(self, on):
        sidp_set_graph(self.ctx, on)

    def synchronize(self):
        sidp_synchronize(self.ctx)

    def tile(self):
        """(tx, ty, index) of the stage kernel's tile candidate (index >= 4: the line kernel)."""
        tx, ty = sidp_get_tile(self.ctx)
        return tx, ty, sidp_get_tile_index(self.ctx)

    def set_tile(self, index):
        sidp_set_tile(self.ctx, index)
