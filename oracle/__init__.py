"""FP64 CPU oracle of the LB / dynamic-IB method (arXiv 2207.06029).

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously correct
statement of what the method computes (``lbib_oracle.c``, built with gcc,
``-O2 -ffp-contract=off``) and a ctypes wrapper around it.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The CUDA library never imports, links or calls it, and it never
imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_WALL = 0, 1
EBODY_WALL = -5

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class BodyParams(C.Structure):
    _fields_ = [("rigid", C.c_int),
                ("ks0", C.c_double), ("Eb", C.c_double), ("kv", C.c_double),
                ("thickness", C.c_double), ("density_ratio", C.c_double),
                ("ref_radius", C.c_double),
                ("gravity", C.c_double * 3), ("u0", C.c_double * 3), ("omega0", C.c_double * 3),
                ("bend_variant", C.c_int), ("kinematic", C.c_int), ("rigid_force", C.c_int),
                ("centroid_markers", C.c_int), ("mass_model", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_lattice.argtypes = [_ip, _dp]
            L.orc_feq.argtypes = [C.c_double, _dp, _dp]
            L.orc_guo.argtypes = [_dp, _dp, C.c_double, _dp]
            L.orc_collide.argtypes = [_dp, C.c_double, _dp, _dp, _dp]
            L.orc_zouhe_face.argtypes = [_dp, C.c_int, C.c_int, _dp]
            L.orc_wall_multi.argtypes = [_dp, C.c_int, _ip, _ip, _dp]
            L.orc_mls_point.argtypes = [_dp, _ip, _dp]
            L.orc_mls_point.restype = C.c_int
            L.orc_volume.argtypes = [_dp, C.c_int, _ip]
            L.orc_volume.restype = C.c_double
            L.orc_area.argtypes = [_dp, C.c_int, _ip]
            L.orc_area.restype = C.c_double
            L.orc_mesh_hinges.argtypes = [C.c_int, C.c_int, _ip, _ip, C.c_void_p]
            L.orc_mesh_hinges.restype = C.c_int
            L.orc_spring_forces.argtypes = [_dp, C.c_int, _ip, _dp, _dp, _dp]
            L.orc_spring_forces.restype = C.c_double
            L.orc_hinge_theta.argtypes = [_dp, _dp, _dp, _dp, C.c_void_p]
            L.orc_hinge_theta.restype = C.c_double
            L.orc_bend_forces.argtypes = [_dp, C.c_int, _ip, _dp, _dp, C.c_int, _dp]
            L.orc_bend_forces.restype = C.c_double
            L.orc_volume_forces.argtypes = [_dp, C.c_int, _ip, C.c_double, C.c_double, _dp]
            L.orc_volume_forces.restype = C.c_double
            L.orc_mass_properties.argtypes = [_dp, C.c_int, _ip, _dp, _dp, _dp]
            L.orc_bdf2.argtypes = [_dp, _dp, _dp, _dp]
            L.orc_verlet.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_sim_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _dp, _ip, _dp]
            L.orc_sim_create.restype = C.c_void_p
            L.orc_sim_destroy.argtypes = [C.c_void_p]
            L.orc_sim_set_fields.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_sim_set_populations.argtypes = [C.c_void_p, _dp]
            L.orc_sim_get_populations.argtypes = [C.c_void_p, _dp]
            L.orc_sim_get_fields.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_sim_add_body.argtypes = [C.c_void_p, _dp, C.c_int, _ip, C.c_int, C.POINTER(BodyParams)]
            L.orc_sim_add_body.restype = C.c_int
            L.orc_sim_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_sim_step.restype = C.c_int
            L.orc_sim_get_markers.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_sim_get_markers.restype = C.c_int
            L.orc_sim_get_body.argtypes = [C.c_void_p, C.c_int, _dp]
            L.orc_sim_get_body.restype = C.c_int
            L.orc_sim_body_rest.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_sim_body_rest.restype = C.c_int
            L.orc_sim_predict.argtypes = [C.c_void_p]
            L.orc_sim_get_predictor.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_sim_get_fib.argtypes = [C.c_void_p, _dp]
            L.orc_hydro_force_fields.argtypes = [_ip, _ip, C.c_double, _dp, _dp, _dp, _ip, _dp, C.c_void_p]
            L.orc_hydro_force_fields.restype = C.c_int
            L.orc_sim_step_count.argtypes = [C.c_void_p]
            L.orc_sim_step_count.restype = C.c_long
    return _lib


def _d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---- single-node and single-element functions -------------------------------------

def lattice():
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    lib().orc_lattice(e, w)
    return e, w


def feq(rho, u):
    out = np.zeros(19)
    lib().orc_feq(float(rho), _d(u, 3), out)
    return out


def guo(u, flb, tau):
    out = np.zeros(19)
    lib().orc_guo(_d(u, 3), _d(flb, 3), float(tau), out)
    return out


def collide(f, tau, flb):
    f = _d(f, 19).copy()
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().orc_collide(f, float(tau), _d(flb, 3), rho, u)
    return f, rho[0], u


def zouhe_face(f, axis, sign, uw):
    f = _d(f, 19).copy()
    lib().orc_zouhe_face(f, int(axis), int(sign), _d(uw, 3))
    return f


def wall_multi(f, axes, signs, uw_faces):
    f = _d(f, 19).copy()
    lib().orc_wall_multi(f, len(axes), _i(axes), _i(signs), _d(uw_faces, 3 * len(axes)))
    return f


def mls_point(X):
    base = np.zeros(3, np.int32)
    psi = np.zeros((27, 4))
    rc = lib().orc_mls_point(_d(X, 3), base, psi)
    if rc:
        raise ValueError("singular MLS moment matrix")
    return base, psi


def mesh_hinges(nv, tris):
    tris = _i(tris)
    nt = tris.shape[0]
    h = np.zeros((3 * nt, 4), np.int32)
    ht = np.zeros((3 * nt, 2), np.int32)
    nh = lib().orc_mesh_hinges(int(nv), nt, tris, h, _ptr(ht))
    if nh < 0:
        raise ValueError("mesh is not a closed oriented manifold")
    return h[:nh].copy(), ht[:nh].copy()


def volume(X, tris):
    tris = _i(tris)
    return lib().orc_volume(_d(X), tris.shape[0], tris)


def area(X, tris):
    tris = _i(tris)
    return lib().orc_area(_d(X), tris.shape[0], tris)


def spring_forces(X, edges, ks, l0):
    X = _d(X)
    F = np.zeros_like(X)
    edges = _i(edges)
    E = lib().orc_spring_forces(X, edges.shape[0], edges, _d(ks), _d(l0), F)
    return E, F


def hinge_theta(xa, xb, xc, xd, with_grad=False):
    g = np.zeros(12)
    th = lib().orc_hinge_theta(_d(xa, 3), _d(xb, 3), _d(xc, 3), _d(xd, 3), _ptr(g) if with_grad else None)
    return (th, g.reshape(4, 3)) if with_grad else th


def bend_forces(X, hinges, kb, theta0, variant=0):
    X = _d(X)
    F = np.zeros_like(X)
    hinges = _i(hinges)
    E = lib().orc_bend_forces(X, hinges.shape[0], hinges, _d(kb), _d(theta0), int(variant), F)
    return E, F


def volume_forces(X, tris, kv, V0):
    X = _d(X)
    F = np.zeros_like(X)
    tris = _i(tris)
    E = lib().orc_volume_forces(X, tris.shape[0], tris, float(kv), float(V0), F)
    return E, F


def mass_properties(X, tris):
    tris = _i(tris)
    V = np.zeros(1)
    c = np.zeros(3)
    I = np.zeros(9)
    lib().orc_mass_properties(_d(X), tris.shape[0], tris, V, c, I)
    return V[0], c, I.reshape(3, 3)


def bdf2(v1, v2, vdot):
    out = np.zeros(3)
    lib().orc_bdf2(_d(v1, 3), _d(v2, 3), _d(vdot, 3), out)
    return out


def verlet(x, xprev, U, acc):
    xn = np.zeros(3)
    un = np.zeros(3)
    lib().orc_verlet(_d(x, 3), _d(xprev, 3), _d(U, 3), _d(acc, 3), xn, un)
    return xn, un


def hydro_force_fields(n, bc, nu, rho, u, X, tri):
    """Pressure + viscous jump force on triangle `tri` of mesh X for nodal
    fields rho (ncell,) and u (ncell, 3) on a lattice of size n."""
    F = np.zeros(3)
    rc = lib().orc_hydro_force_fields(_i(n), _i(bc), float(nu), _d(rho), _d(u), _d(X), _i(tri), F, None)
    if rc:
        raise ValueError(f"probe support reaches a wall ({rc})")
    return F


# ---- whole-method simulation --------------------------------------------------------

class Sim:
    """Oracle simulation: the lattice, its walls and the immersed bodies."""

    def __init__(self, n, tau, gext=(0, 0, 0), bc=(BC_PERIODIC,) * 3, wall_u=None):
        self.n = tuple(int(v) for v in n)
        wall = np.zeros((6, 3)) if wall_u is None else _d(wall_u).reshape(6, 3)
        self._h = lib().orc_sim_create(self.n[0], self.n[1], self.n[2], float(tau), _d(gext, 3),
                                       _i(bc), _d(wall.ravel()))
        if not self._h:
            raise ValueError("invalid lattice parameters")
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.nv = []

    def close(self):
        if self._h:
            lib().orc_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho, u):
        lib().orc_sim_set_fields(self._h, _d(rho, self.ncell), _d(u, 3 * self.ncell))

    def set_populations(self, f):
        lib().orc_sim_set_populations(self._h, _d(f, 19 * self.ncell))

    def populations(self):
        """Post-collision populations, shape (ncell, 19), x fastest in ncell."""
        f = np.zeros(19 * self.ncell)
        lib().orc_sim_get_populations(self._h, f)
        return f.reshape(self.ncell, 19)

    def fields(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        lib().orc_sim_get_fields(self._h, rho, u)
        return rho, u.reshape(self.ncell, 3)

    def predictor(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        lib().orc_sim_get_predictor(self._h, rho, u)
        return rho, u.reshape(self.ncell, 3)

    def fib(self):
        f = np.zeros(3 * self.ncell)
        lib().orc_sim_get_fib(self._h, f)
        return f.reshape(self.ncell, 3)

    def add_body(self, verts, tris, *, rigid=False, ks0=0.0, Eb=0.0, kv=0.0, thickness=1.0,
                 density_ratio=1.0, ref_radius=1.0, gravity=(0, 0, 0), u0=(0, 0, 0), omega0=(0, 0, 0),
                 bend_variant=0, kinematic=0, rigid_force=0, centroid_markers=0, mass_model=0):
        verts = _d(verts)
        tris = _i(tris)
        p = BodyParams(int(rigid), ks0, Eb, kv, thickness, density_ratio, ref_radius,
                       (C.c_double * 3)(*gravity), (C.c_double * 3)(*u0), (C.c_double * 3)(*omega0),
                       int(bend_variant), int(kinematic), int(rigid_force), int(centroid_markers), int(mass_model))
        bid = lib().orc_sim_add_body(self._h, verts, verts.shape[0], tris, tris.shape[0], C.byref(p))
        if bid < 0:
            raise ValueError(f"orc_sim_add_body failed ({bid})")
        self.nv.append(verts.shape[0])
        return bid

    def step(self, n=1):
        return lib().orc_sim_step(self._h, int(n))

    def predict(self):
        lib().orc_sim_predict(self._h)

    def markers(self, body=0):
        nv = self.nv[body]
        X = np.zeros((nv, 3))
        V = np.zeros((nv, 3))
        F = np.zeros((nv, 3))
        rc = lib().orc_sim_get_markers(self._h, body, _ptr(X), _ptr(V), _ptr(F))
        if rc:
            raise ValueError("bad body")
        return X, V, F

    def body(self, body=0):
        out = np.zeros(15)
        lib().orc_sim_get_body(self._h, body, out)
        return {"xc": out[0:3], "u": out[3:6], "omega": out[6:9], "q": out[9:13],
                "volume": out[13], "area": out[14]}

    def body_rest(self, body=0):
        nh = self.nv[body] * 3  # upper bound: E = 3V - 6 for a closed genus-0 mesh
        h = np.zeros((nh, 4), np.int32)
        ks, l0, kb, th0 = (np.zeros(nh) for _ in range(4))
        sc = np.zeros(5)
        n = lib().orc_sim_body_rest(self._h, body, _ptr(h), _ptr(ks), _ptr(l0), _ptr(kb), _ptr(th0), _ptr(sc))
        return {"hinge": h[:n], "ks": ks[:n], "l0": l0[:n], "kb": kb[:n], "theta0": th0[:n],
                "V0": sc[0], "A0": sc[1], "mv": sc[2], "m": sc[3], "Vb": sc[4]}

    @property
    def step_count(self):
        return lib().orc_sim_step_count(self._h)
