"""ctypes binding of liblbib (C ABI in include/lbib.h), with the same names.

Argument marshalling only: every step of the method runs in the CUDA
library.  If the library is missing, importing a function raises
``RuntimeError`` (there is no CPU fallback).  Arrays may be numpy arrays
(host) or torch CUDA tensors (device, passed with ``on_device=1``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbib.so")

LBIB_OK, LBIB_EINVAL, LBIB_ENOMEM, LBIB_ECUDA, LBIB_EDIVERGED, LBIB_EBODY_WALL, LBIB_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LBIB_ETOOBIG = -7
LBIB_NOALLOC_MAX_TRIS = 1 << 20
LBIB_FP64, LBIB_FP32, LBIB_FP16_DEV, LBIB_BF16_DEV = 0, 1, 2, 3
LBIB_PERIODIC, LBIB_WALL = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbib_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("body_force", C.c_double * 3),
                ("bc", C.c_int * 3), ("wall_u", (C.c_double * 3) * 6),
                ("precision", C.c_int), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class lbib_body_params(C.Structure):
    _fields_ = [("rigid", C.c_int), ("ks0", C.c_double), ("Eb", C.c_double), ("kv", C.c_double),
                ("thickness", C.c_double), ("density_ratio", C.c_double), ("ref_radius", C.c_double),
                ("gravity", C.c_double * 3), ("u0", C.c_double * 3), ("omega0", C.c_double * 3),
                ("bend_variant", C.c_int), ("kinematic", C.c_int), ("rigid_force", C.c_int),
                ("centroid_markers", C.c_int), ("mass_model", C.c_int)]


class lbib_body_state(C.Structure):
    _fields_ = [("xc", C.c_double * 3), ("u", C.c_double * 3), ("omega", C.c_double * 3),
                ("q", C.c_double * 4), ("volume", C.c_double), ("area", C.c_double)]


LBIB_REQ_QUEUED, LBIB_REQ_RUNNING, LBIB_REQ_DONE, LBIB_REQ_FAILED = 0, 1, 2, 3
LBIB_SERVE_BATCHED, LBIB_SERVE_PLAIN = 0, 1
LBIB_SERVE_SHORTEST, LBIB_SERVE_OLDEST = 0, 1


class lbib_serve_params(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("chunk_steps", C.c_int), ("max_active", C.c_int), ("mode", C.c_int),
                ("batch_cells", C.c_longlong), ("batch_order", C.c_int)]


class lbib_serve_times(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("queued_s", C.c_double), ("latency_s", C.c_double),
                ("done_s", C.c_double), ("error", C.c_char * 160)]


class lbib_serve_summary(C.Structure):
    _fields_ = [("runs_done", C.c_longlong), ("runs_failed", C.c_longlong), ("queued", C.c_longlong),
                ("active", C.c_longlong), ("chunks", C.c_longlong), ("rebuilds", C.c_longlong),
                ("cell_updates", C.c_double), ("busy_s", C.c_double), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t)]


class LbibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbib error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

EXPORTS = ["lbib_create", "lbib_set_fields", "lbib_set_shear_fields", "lbib_set_populations", "lbib_add_body", "lbib_step", "lbib_sync",
           "lbib_set_watchdog", "lbib_check",
           "lbib_get_fields", "lbib_get_populations", "lbib_get_totals", "lbib_get_markers", "lbib_get_markers_async", "lbib_step_markers", "lbib_get_body", "lbib_counters",
           "lbib_profile", "lbib_get_profile", "lbib_set_output", "lbib_set_overlap", "lbib_set_graphs", "lbib_set_sweep_config", "lbib_autotune",
           "lbib_set_ib_blocks", "lbib_get_launch_config",
           "lbib_device_bytes", "lbib_save", "lbib_load", "lbib_mesh_measures_noalloc",
           "lbib_batch_create", "lbib_batch_step", "lbib_batch_sync", "lbib_batch_counters", "lbib_batch_autotune",
           "lbib_batch_set_config", "lbib_batch_set_persistent",
           "lbib_batch_destroy", "lbib_batch_last_error",
           "lbib_request_create", "lbib_request_add_body", "lbib_request_destroy", "lbib_serve_create",
           "lbib_serve_submit", "lbib_serve_wait", "lbib_serve_take", "lbib_serve_stats", "lbib_serve_destroy",
           "lbib_measure_fma", "lbib_destroy",
           "lbib_last_error"]


def load():
    """Loads liblbib.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblbib.so not found at {LIB_PATH}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.lbib_create.argtypes = [C.POINTER(lbib_params), C.POINTER(C.c_void_p)]
        L.lbib_set_fields.argtypes = [vp, vp, vp, C.c_int]
        L.lbib_set_populations.argtypes = [vp, vp, C.c_int]
        L.lbib_add_body.argtypes = [vp, vp, C.c_int, vp, C.c_int, C.POINTER(lbib_body_params), ip]
        L.lbib_step.argtypes = [vp, C.c_int]
        L.lbib_sync.argtypes = [vp]
        L.lbib_set_watchdog.argtypes = [vp, C.c_int, C.c_double]
        L.lbib_check.argtypes = [vp]
        L.lbib_get_fields.argtypes = [vp, vp, vp, C.c_int]
        L.lbib_get_populations.argtypes = [vp, vp, C.c_int]
        L.lbib_get_totals.argtypes = [vp, dp]
        L.lbib_get_markers.argtypes = [vp, C.c_int, vp, vp, vp]
        L.lbib_get_markers_async.argtypes = [vp, C.c_int, vp, vp, vp]
        L.lbib_measure_fma.argtypes = [C.c_int, dp]
        L.lbib_step_markers.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
        L.lbib_get_body.argtypes = [vp, C.c_int, C.POINTER(lbib_body_state)]
        L.lbib_counters.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.lbib_profile.argtypes = [vp, C.c_int]
        L.lbib_get_profile.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
        L.lbib_set_output.argtypes = [vp, C.c_int]
        L.lbib_set_overlap.argtypes = [vp, C.c_int]
        L.lbib_set_graphs.argtypes = [vp, C.c_int]
        L.lbib_set_sweep_config.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.lbib_set_ib_blocks.argtypes = [vp, C.c_int]
        L.lbib_set_shear_fields.argtypes = [vp, C.c_double, C.c_double]
        L.lbib_get_launch_config.argtypes = [vp, ip]
        L.lbib_autotune.argtypes = [vp, C.c_int, ip]
        L.lbib_device_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.lbib_save.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.lbib_load.argtypes = [vp, vp, C.c_size_t]
        L.lbib_mesh_measures_noalloc.argtypes = [vp, C.c_int, vp, C.c_int, vp, vp]
        L.lbib_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, vp, C.POINTER(C.c_void_p)]
        L.lbib_batch_step.argtypes = [vp, C.c_int]
        L.lbib_batch_sync.argtypes = [vp]
        L.lbib_batch_counters.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.lbib_batch_autotune.argtypes = [vp, C.c_int, ip]
        L.lbib_batch_set_config.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.lbib_batch_set_persistent.argtypes = [vp, C.c_int, C.c_double]
        L.lbib_batch_destroy.argtypes = [vp]
        L.lbib_batch_destroy.restype = None
        L.lbib_batch_last_error.argtypes = [vp]
        L.lbib_batch_last_error.restype = C.c_char_p
        L.lbib_request_create.argtypes = [C.POINTER(lbib_params), C.c_longlong, C.c_int, C.POINTER(C.c_void_p)]
        L.lbib_request_add_body.argtypes = [vp, vp, C.c_int, vp, C.c_int, C.POINTER(lbib_body_params)]
        L.lbib_request_destroy.argtypes = [vp]
        L.lbib_request_destroy.restype = None
        L.lbib_serve_create.argtypes = [C.POINTER(lbib_serve_params), C.POINTER(C.c_void_p)]
        L.lbib_serve_submit.argtypes = [vp, vp, C.POINTER(C.c_longlong)]
        L.lbib_serve_wait.argtypes = [vp, C.c_longlong, C.c_double, ip]
        L.lbib_serve_take.argtypes = [vp, C.c_longlong, C.POINTER(C.c_void_p), C.POINTER(lbib_serve_times)]
        L.lbib_serve_stats.argtypes = [vp, C.POINTER(lbib_serve_summary)]
        L.lbib_serve_destroy.argtypes = [vp]
        L.lbib_serve_destroy.restype = None
        L.lbib_destroy.argtypes = [vp]
        L.lbib_destroy.restype = None
        L.lbib_last_error.argtypes = [vp]
        L.lbib_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("lbib_destroy", "lbib_last_error", "lbib_batch_destroy", "lbib_batch_last_error",
                            "lbib_request_destroy", "lbib_serve_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(ctx, rc):
    if rc != LBIB_OK:
        msg = load().lbib_last_error(ctx)
        raise LbibError(rc, msg.decode() if msg else "")
    return rc


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    """Host numpy array or CUDA tensor -> (pointer, on_device)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    return a.ctypes.data_as(C.c_void_p), 0


# ---- thin wrappers with the ABI names ------------------------------------------------

def lbib_create(params: lbib_params):
    h = C.c_void_p()
    rc = load().lbib_create(C.byref(params), C.byref(h))
    _check(None, rc)
    return h


def lbib_set_fields(ctx, rho, u):
    pr, dev = _ptr(rho)
    pu, _ = _ptr(u)
    return _check(ctx, load().lbib_set_fields(ctx, pr, pu, dev))


def lbib_set_populations(ctx, f):
    pf, dev = _ptr(f)
    return _check(ctx, load().lbib_set_populations(ctx, pf, dev))


def lbib_add_body(ctx, verts, tris, bp: lbib_body_params):
    verts = _host(verts, np.float64)
    tris = _host(tris, np.int32)
    bid = C.c_int(-1)
    _check(ctx, load().lbib_add_body(ctx, verts.ctypes.data_as(C.c_void_p), verts.shape[0],
                                     tris.ctypes.data_as(C.c_void_p), tris.shape[0], C.byref(bp), C.byref(bid)))
    return bid.value


def lbib_step(ctx, nsteps):
    return _check(ctx, load().lbib_step(ctx, int(nsteps)))


def lbib_sync(ctx):
    return _check(ctx, load().lbib_sync(ctx))


def lbib_set_watchdog(ctx, every, mass_tol=0.1):
    return _check(ctx, load().lbib_set_watchdog(ctx, int(every), float(mass_tol)))


def lbib_check(ctx):
    return _check(ctx, load().lbib_check(ctx))


def lbib_get_fields(ctx, rho, u):
    pr, dev = _ptr(rho)
    pu, dev2 = _ptr(u)
    return _check(ctx, load().lbib_get_fields(ctx, pr, pu, max(dev, dev2)))


def lbib_get_totals(ctx):
    """(mass, momentum[3]) of the populations, reduced on the GPU in FP64."""
    out = (C.c_double * 4)()
    _check(ctx, load().lbib_get_totals(ctx, out))
    return out[0], np.array(out[1:4])


def lbib_get_populations(ctx, f):
    pf, dev = _ptr(f)
    return _check(ctx, load().lbib_get_populations(ctx, pf, dev))


def lbib_get_markers(ctx, body, X=None, V=None, F=None):
    return _check(ctx, load().lbib_get_markers(ctx, int(body), _ptr(X)[0], _ptr(V)[0], _ptr(F)[0]))


def lbib_get_markers_async(ctx, body, X=None, V=None, F=None):
    """Queues the copies (host arrays or page-locked CPU tensors; read them
    after a synchronisation)."""
    return _check(ctx, load().lbib_get_markers_async(ctx, int(body), _ptr(X)[0], _ptr(V)[0], _ptr(F)[0]))


def lbib_step_markers(ctx, nsteps, body, X=None, V=None, F=None):
    """nsteps steps, the markers of each queued for copying into X[k], V[k],
    F[k] (arrays of shape (nsteps, nv, 3); read them after a
    synchronisation)."""
    return _check(ctx, load().lbib_step_markers(ctx, int(nsteps), int(body), _ptr(X)[0], _ptr(V)[0], _ptr(F)[0]))


def lbib_measure_fma(fp64=True):
    """FMA throughput of the current device in flops/s (a measurement aid)."""
    out = C.c_double()
    rc = load().lbib_measure_fma(int(bool(fp64)), C.byref(out))
    _check(None, rc)
    return out.value


def lbib_get_body(ctx, body):
    st = lbib_body_state()
    _check(ctx, load().lbib_get_body(ctx, int(body), C.byref(st)))
    return st


def lbib_counters(ctx):
    s, l = C.c_longlong(), C.c_longlong()
    _check(ctx, load().lbib_counters(ctx, C.byref(s), C.byref(l)))
    return s.value, l.value


def lbib_profile(ctx, enable):
    return _check(ctx, load().lbib_profile(ctx, int(enable)))


def lbib_get_profile(ctx):
    """Returns (mls_ms, structure_ms, sweep_ms, step_ms, nsteps) accumulated since the last read."""
    ms = (C.c_double * 4)()
    n = C.c_longlong()
    _check(ctx, load().lbib_get_profile(ctx, ms, C.byref(n)))
    return ms[0], ms[1], ms[2], ms[3], n.value


def lbib_autotune(ctx, steps):
    """Returns (block_x, block_y, overlap, row_tiles, far_per_sm) chosen; advances the run by several
    times `steps`."""
    ch = (C.c_int * 5)()
    _check(ctx, load().lbib_autotune(ctx, int(steps), ch))
    return tuple(ch)


def lbib_set_overlap(ctx, enable):
    return _check(ctx, load().lbib_set_overlap(ctx, int(enable)))


def lbib_save(ctx):
    """Checkpoint of the context as bytes."""
    n = C.c_size_t(0)
    _check(ctx, load().lbib_save(ctx, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, load().lbib_save(ctx, buf, C.byref(n)))
    return buf.raw[:n.value]


def lbib_load(ctx, data):
    buf = C.create_string_buffer(bytes(data), len(data))
    return _check(ctx, load().lbib_load(ctx, buf, len(data)))


def lbib_set_sweep_config(ctx, row_tiles, block_x=0, block_y=0, far_per_sm=0):
    return _check(ctx, load().lbib_set_sweep_config(ctx, int(row_tiles), int(block_x), int(block_y),
                                                    int(far_per_sm)))


def lbib_set_shear_fields(ctx, u_lo, u_hi):
    return _check(ctx, load().lbib_set_shear_fields(ctx, float(u_lo), float(u_hi)))


def lbib_set_ib_blocks(ctx, per_sm):
    return _check(ctx, load().lbib_set_ib_blocks(ctx, int(per_sm)))


def lbib_get_launch_config(ctx):
    """(block_x, block_y, overlap, row_tiles, far_per_sm, ib_per_sm) in use."""
    cfg = (C.c_int * 6)()
    _check(ctx, load().lbib_get_launch_config(ctx, cfg))
    return tuple(cfg)


def lbib_set_graphs(ctx, enable):
    return _check(ctx, load().lbib_set_graphs(ctx, int(enable)))


def lbib_set_output(ctx, fields_every):
    return _check(ctx, load().lbib_set_output(ctx, int(fields_every)))


def lbib_device_bytes(ctx):
    n = C.c_size_t()
    _check(ctx, load().lbib_device_bytes(ctx, C.byref(n)))
    return n.value


def lbib_destroy(ctx):
    load().lbib_destroy(ctx)


def lbib_last_error(ctx):
    m = load().lbib_last_error(ctx)
    return m.decode() if m else ""


# ---- convenience object used by tests and the benchmark ------------------------------

def make_params(n, tau, *, bc=(0, 0, 0), wall_u=None, body_force=(0, 0, 0), precision=LBIB_FP32, stream=None):
    p = lbib_params()
    p.nx, p.ny, p.nz = (int(v) for v in n)
    p.tau = float(tau)
    for a in range(3):
        p.body_force[a] = float(body_force[a])
        p.bc[a] = int(bc[a])
    w = np.zeros((6, 3)) if wall_u is None else np.asarray(wall_u, np.float64).reshape(6, 3)
    for f in range(6):
        for a in range(3):
            p.wall_u[f][a] = float(w[f, a])
    p.precision = int(precision)
    p.stream = stream
    return p


def make_body_params(*, rigid=False, ks0=0.0, Eb=0.0, kv=0.0, thickness=1.0, density_ratio=1.0, ref_radius=1.0,
                     gravity=(0, 0, 0), u0=(0, 0, 0), omega0=(0, 0, 0), bend_variant=0, kinematic=0, rigid_force=0,
                     centroid_markers=0, mass_model=0):
    bp = lbib_body_params()
    bp.rigid = int(rigid)
    bp.ks0, bp.Eb, bp.kv = float(ks0), float(Eb), float(kv)
    bp.thickness, bp.density_ratio, bp.ref_radius = float(thickness), float(density_ratio), float(ref_radius)
    for a in range(3):
        bp.gravity[a] = float(gravity[a])
        bp.u0[a] = float(u0[a])
        bp.omega0[a] = float(omega0[a])
    bp.bend_variant = int(bend_variant)
    bp.kinematic = int(kinematic)
    bp.rigid_force = int(rigid_force)
    bp.centroid_markers = int(centroid_markers)
    bp.mass_model = int(mass_model)
    return bp


class Context:
    """One lattice with its bodies on the GPU."""

    def __init__(self, n, tau, *, bc=(0, 0, 0), wall_u=None, body_force=(0, 0, 0), precision=LBIB_FP32,
                 stream=None):
        self.n = tuple(int(v) for v in n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.h = lbib_create(make_params(n, tau, bc=bc, wall_u=wall_u, body_force=body_force,
                                         precision=precision, stream=stream))
        self.nv = []

    @classmethod
    def adopt(cls, h, n, nv):
        """Wraps an existing context handle (e.g. one taken from a server):
        lattice dims n and the vertex count of each body."""
        ctx = cls.__new__(cls)
        ctx.n = tuple(int(v) for v in n)
        ctx.ncell = ctx.n[0] * ctx.n[1] * ctx.n[2]
        ctx.h = h
        ctx.nv = [int(v) for v in nv]
        return ctx

    @classmethod
    def from_case(cls, case, precision=None, stream=None):
        ctx = cls(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, body_force=case.gext,
                  precision=case.precision if precision is None else precision, stream=stream)
        rho, u = case.initial_fields()
        ctx.set_fields(rho, u)
        for b in case.bodies:
            ctx.add_body(b.verts, b.tris, **b.kwargs())
        return ctx

    def close(self):
        if getattr(self, "h", None):
            lbib_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho, u):
        lbib_set_fields(self.h, _host(rho, np.float64), _host(u, np.float64).reshape(-1))

    def set_populations(self, f):
        lbib_set_populations(self.h, _host(f, np.float64).reshape(-1))

    def add_body(self, verts, tris, **kw):
        bid = lbib_add_body(self.h, verts, tris, make_body_params(**kw))
        self.nv.append(int(np.asarray(verts).shape[0]))
        return bid

    def step(self, n=1):
        lbib_step(self.h, n)

    def sync(self):
        lbib_sync(self.h)

    def fields(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        lbib_get_fields(self.h, rho, u)
        return rho, u.reshape(self.ncell, 3)

    def populations(self):
        f = np.zeros(19 * self.ncell)
        lbib_get_populations(self.h, f)
        return f.reshape(self.ncell, 19)

    def markers(self, body=0):
        nv = self.nv[body]
        X, V, F = (np.zeros((nv, 3)) for _ in range(3))
        lbib_get_markers(self.h, body, X, V, F)
        return X, V, F

    def body(self, body=0):
        st = lbib_get_body(self.h, body)
        return {"xc": np.array(st.xc), "u": np.array(st.u), "omega": np.array(st.omega), "q": np.array(st.q),
                "volume": st.volume, "area": st.area}

    def counters(self):
        return lbib_counters(self.h)


_NOALLOC_MESSAGES = {
    LBIB_ETOOBIG: f"more than LBIB_NOALLOC_MAX_TRIS = {LBIB_NOALLOC_MAX_TRIS} triangles",
    LBIB_EINVAL: "negative size or NULL array",
    LBIB_ECUDA: "a CUDA call failed (device lookup of the scratch array or the launch)",
}


CUDA_STREAM_PER_THREAD = 2  # cudaStreamPerThread


def lbib_mesh_measures_noalloc(X, nv, tris, nt, out, stream=CUDA_STREAM_PER_THREAD):
    """Volume and area of a closed mesh into out[2], allocating nothing.
    X (nv x 3 float64), tris (nt x 3 int32) and out (2 float64) are CUDA
    tensors on the current device, contiguous, or raw device pointers
    (ints, unchecked).  stream is a cudaStream_t handle (int); the default
    is the per-thread default stream, which never synchronises implicitly
    with other streams (None passes NULL, the legacy default stream)."""
    import torch
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None

    def addr(a, dtype, name):
        if not hasattr(a, "data_ptr"):
            return C.c_void_p(a)
        if a.dtype != dtype or not a.is_cuda or not a.is_contiguous() or a.device.index != dev:
            raise LbibError(LBIB_EINVAL, f"{name} must be a contiguous {dtype} CUDA tensor on device {dev} "
                                         f"(got {a.dtype}, {a.device}, contiguous={a.is_contiguous()})")
        return C.c_void_p(a.data_ptr())
    pX = addr(X, torch.float64, "X")
    pT = addr(tris, torch.int32, "tris")
    pO = addr(out, torch.float64, "out")
    if hasattr(X, "numel") and X.numel() < 3 * int(nv):
        raise LbibError(LBIB_EINVAL, f"X holds {X.numel()} values, fewer than 3 * nv = {3 * int(nv)}")
    if hasattr(tris, "numel") and int(nt) > 0 and tris.numel() < 3 * int(nt):
        raise LbibError(LBIB_EINVAL, f"tris holds {tris.numel()} values, fewer than 3 * nt = {3 * int(nt)}")
    if hasattr(out, "numel") and out.numel() < 2:
        raise LbibError(LBIB_EINVAL, "out must hold 2 values")
    rc = load().lbib_mesh_measures_noalloc(pX, int(nv), pT, int(nt), pO,
                                           C.c_void_p(stream) if stream else None)
    if rc != LBIB_OK:
        raise LbibError(rc, _NOALLOC_MESSAGES.get(rc, "error"))
    return rc


# ---- batches ---------------------------------------------------------------------------

def _bcheck(batch, rc):
    if rc != LBIB_OK:
        msg = load().lbib_batch_last_error(batch)
        raise LbibError(rc, msg.decode() if msg else "")
    return rc


def lbib_batch_create(ctxs, stream=None):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    h = C.c_void_p()
    _bcheck(None, load().lbib_batch_create(arr, len(ctxs), C.c_void_p(stream) if stream else None, C.byref(h)))
    return h


def lbib_batch_step(batch, nsteps):
    return _bcheck(batch, load().lbib_batch_step(batch, int(nsteps)))


def lbib_batch_sync(batch):
    return _bcheck(batch, load().lbib_batch_sync(batch))


def lbib_batch_counters(batch):
    s, l = C.c_longlong(), C.c_longlong()
    _bcheck(batch, load().lbib_batch_counters(batch, C.byref(s), C.byref(l)))
    return s.value, l.value


def lbib_batch_autotune(batch, steps):
    """(threads per sweep block, lattice order, cells per sweep thread) chosen."""
    ch = (C.c_int * 3)()
    _bcheck(batch, load().lbib_batch_autotune(batch, int(steps), ch))
    return tuple(ch)


def lbib_batch_set_persistent(batch, enable, wait_limit_s=2.0):
    return _bcheck(batch, load().lbib_batch_set_persistent(batch, int(enable), float(wait_limit_s)))


def lbib_batch_set_config(batch, threads, order, cells_per_thread):
    _bcheck(batch, load().lbib_batch_set_config(batch, int(threads), int(order), int(cells_per_thread)))


def lbib_batch_destroy(batch):
    load().lbib_batch_destroy(batch)


def lbib_batch_last_error(batch):
    m = load().lbib_batch_last_error(batch)
    return m.decode() if m else ""


class Batch:
    """Several contexts advanced by common launches."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        self.h = lbib_batch_create([c.h for c in self.contexts], stream)

    def step(self, n=1):
        lbib_batch_step(self.h, n)

    def sync(self):
        lbib_batch_sync(self.h)

    def autotune(self, steps=5):
        return lbib_batch_autotune(self.h, steps)

    def set_config(self, threads, order, cells_per_thread):
        lbib_batch_set_config(self.h, threads, order, cells_per_thread)

    def set_persistent(self, enable, wait_limit_s=2.0):
        lbib_batch_set_persistent(self.h, enable, wait_limit_s)

    def counters(self):
        return lbib_batch_counters(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbib_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving ---------------------------------------------------------------------------

def _scheck(rc, what):
    if rc != LBIB_OK:
        raise LbibError(rc, what)
    return rc


def lbib_request_create(params, nsteps, init=0):
    h = C.c_void_p()
    _scheck(load().lbib_request_create(C.byref(params), int(nsteps), int(init), C.byref(h)), "request")
    return h


def lbib_request_add_body(req, verts, tris, bp):
    v = _host(verts, np.float64).reshape(-1, 3)
    t = _host(tris, np.int32).reshape(-1, 3)
    return _scheck(load().lbib_request_add_body(req, v.ctypes.data_as(C.c_void_p), v.shape[0],
                                                t.ctypes.data_as(C.c_void_p), t.shape[0], C.byref(bp)), "request body")


def lbib_request_destroy(req):
    load().lbib_request_destroy(req)


def lbib_serve_create(hbm_budget, chunk_steps=500, max_active=64, mode=LBIB_SERVE_BATCHED, batch_cells=0,
                      batch_order=0):
    sp = lbib_serve_params(int(hbm_budget), int(chunk_steps), int(max_active), int(mode), int(batch_cells),
                           int(batch_order))
    h = C.c_void_p()
    _scheck(load().lbib_serve_create(C.byref(sp), C.byref(h)), "server")
    return h


def lbib_serve_submit(server, req):
    i = C.c_longlong()
    _scheck(load().lbib_serve_submit(server, req, C.byref(i)), "submit")
    return i.value


def lbib_serve_wait(server, rid, timeout_s=-1.0):
    st = C.c_int()
    rc = load().lbib_serve_wait(server, int(rid), float(timeout_s), C.byref(st))
    return rc, st.value


def lbib_serve_take(server, rid):
    """(context handle or None, times dict, return code)."""
    h = C.c_void_p()
    t = lbib_serve_times()
    rc = load().lbib_serve_take(server, int(rid), C.byref(h), C.byref(t))
    return (h if h.value else None), {"submit_s": t.submit_s, "queued_s": t.queued_s, "latency_s": t.latency_s,
                                      "done_s": t.done_s, "error": t.error.decode(errors="replace")}, rc


def lbib_serve_stats(server):
    s = lbib_serve_summary()
    _scheck(load().lbib_serve_stats(server, C.byref(s)), "stats")
    return {k: getattr(s, k) for k, _ in lbib_serve_summary._fields_}


def lbib_serve_destroy(server):
    load().lbib_serve_destroy(server)


def request_from_case(case, nsteps, precision=None):
    """A request for a workloads.Case: rest or linear-shear initial state
    (the case's initial velocity must be one of the two)."""
    p = make_params(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, body_force=case.gext,
                    precision=case.precision if precision is None else precision)
    init = 0 if case.u0 is None else 1
    req = lbib_request_create(p, nsteps, init)
    for b in case.bodies:
        lbib_request_add_body(req, b.verts, b.tris, make_body_params(**b.kwargs()))
    return req
