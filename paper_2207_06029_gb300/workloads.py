"""Seeded synthetic inputs: immersed-body meshes and the lattice cases.

This module builds inputs only (meshes, initial fields, parameters).  It
holds none of the method's arithmetic and imports neither the CUDA library
nor the oracle, so both sides can take their inputs from it.

The paper's own cases (a sphere settling in a walled box, capsules and
spheroids between two counter-moving walls; Sec. 3.2-3.5) depend on
experimental and literature data that are not available; the cases below
keep their shapes: lattice sizes, relaxation times, surface meshes with
three to five markers per cell, shear rates and density ratios.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

PERIODIC, WALL = 0, 1
PREC_FP64, PREC_FP32, PREC_FP16_DEV, PREC_BF16_DEV = 0, 1, 2, 3


# ---------------------------------------------------------------------------------------
# Meshes
# ---------------------------------------------------------------------------------------

def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _orient_outward(v, f):
    """Make every triangle counter-clockwise seen from outside a star-shaped body."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", n, cen - v.mean(axis=0)) < 0
    f = f.copy()
    f[flip] = f[flip][:, [0, 2, 1]]
    return f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0), axes=None):
    """Unit icosahedron subdivided `level` times (midpoints projected to the
    sphere), scaled to `radius` (or to semi-axes `axes`) and moved to `center`.
    V = 10*4^L + 2 vertices, F = 20*4^L triangles, outward orientation."""
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    faces = [tuple(x) for x in f]
    for _ in range(level):
        cache = {}
        new_faces = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = (np.array(verts[i]) + np.array(verts[j])) / 2.0
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    V = np.array(verts, dtype=np.float64)
    F = np.array(faces, dtype=np.int64)
    F = _orient_outward(V, F)
    if axes is None:
        V = V * float(radius)
    else:
        V = V * np.asarray(axes, dtype=np.float64)[None, :]
    V = V + np.asarray(center, dtype=np.float64)[None, :]
    return np.ascontiguousarray(V), np.ascontiguousarray(F.astype(np.int32))


def cube_mesh(side: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Closed cube of 8 vertices and 12 outward triangles."""
    h = side / 2.0
    v = np.array([[x, y, z] for z in (-h, h) for y in (-h, h) for x in (-h, h)], dtype=np.float64)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    f = _orient_outward(v, np.array(f, dtype=np.int64))
    return v + np.asarray(center)[None, :], f.astype(np.int32)


def perturb(verts, amplitude: float, seed: int):
    rng = np.random.default_rng(seed)
    return verts + amplitude * rng.standard_normal(verts.shape)


# ---------------------------------------------------------------------------------------
# Parameter helpers (inputs derived from dimensionless groups of the paper)
# ---------------------------------------------------------------------------------------

def viscosity(tau: float) -> float:
    """Lattice kinematic viscosity for relaxation time tau (c_s^2 = 1/3)."""
    return (tau - 0.5) / 3.0


def ks0_from_capillary(Ca: float, tau: float, shear_rate: float, radius: float, rho: float = 1.0) -> float:
    """Global membrane stiffness from the capillary number Ca = rho nu u_ref / k_s0
    with u_ref = shear rate x radius (Sec. 2.3 and Sec. 3.4)."""
    return rho * viscosity(tau) * shear_rate * radius / Ca


def settling_gravity(Re: float, gamma: float, d: float, tau: float) -> float:
    """Gravity for a terminal Reynolds number Re = d u_inf / nu at density ratio
    gamma, from Abraham's drag law C_d = C0 (1 + delta0/sqrt(Re))^2 with
    C0 delta0^2 = 24, delta0 = 9.06, and u_inf^2 = 4 g d (gamma - 1) / (3 C_d)
    (Sec. 3.2)."""
    delta0 = 9.06
    C0 = 24.0 / delta0 ** 2
    Cd = C0 * (1.0 + delta0 / math.sqrt(Re)) ** 2
    u_inf = Re * viscosity(tau) / d
    return 3.0 * Cd * u_inf ** 2 / (4.0 * d * (gamma - 1.0))


# ---------------------------------------------------------------------------------------
# Cases
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass
class Body:
    verts: np.ndarray
    tris: np.ndarray
    rigid: bool = False
    ks0: float = 0.0
    Eb: float = 0.0
    kv: float = 0.0
    thickness: float = 1.0
    density_ratio: float = 1.0
    ref_radius: float = 1.0
    gravity: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    u0: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    omega0: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    bend_variant: int = 0
    kinematic: int = 0
    rigid_force: int = 0
    centroid_markers: int = 0
    mass_model: int = 0  # membrane mass: 0 shell of thickness T (Sec. 3.5), 1 capsule of density rho_s (Sec. 3.4)

    def kwargs(self):
        return dict(rigid=self.rigid, ks0=self.ks0, Eb=self.Eb, kv=self.kv, thickness=self.thickness,
                    density_ratio=self.density_ratio, ref_radius=self.ref_radius, gravity=self.gravity,
                    u0=self.u0, omega0=self.omega0, bend_variant=self.bend_variant, kinematic=self.kinematic,
                    rigid_force=self.rigid_force, centroid_markers=self.centroid_markers,
                    mass_model=self.mass_model)


@dataclasses.dataclass
class Case:
    name: str
    n: Tuple[int, int, int]
    tau: float
    bc: Tuple[int, int, int]
    wall_u: np.ndarray                  # (6, 3): faces -x,+x,-y,+y,-z,+z
    gext: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    precision: int = PREC_FP32
    steps: int = 100
    bodies: List[Body] = dataclasses.field(default_factory=list)
    rho0: Optional[np.ndarray] = None   # (ncell,)
    u0: Optional[np.ndarray] = None     # (ncell, 3)

    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]

    def initial_fields(self):
        rho = np.ones(self.ncell) if self.rho0 is None else self.rho0
        u = np.zeros((self.ncell, 3)) if self.u0 is None else self.u0
        return np.ascontiguousarray(rho, np.float64), np.ascontiguousarray(u, np.float64)


def couette_profile(n, U: float):
    """Linear shear u_x(z) = U (2 z/(nz-1) - 1) between walls at z = 0 and nz-1,
    the exact steady state; x fastest in the flattened index."""
    nx, ny, nz = n
    z = np.arange(nz, dtype=np.float64)
    ux = U * (2.0 * z / (nz - 1) - 1.0)
    u = np.zeros((nz, ny, nx, 3))
    u[..., 0] = ux[:, None, None]
    return u.reshape(-1, 3)


def shear_walls(U: float):
    w = np.zeros((6, 3))
    w[4, 0] = -U   # z = 0 face moves along -x
    w[5, 0] = +U   # z = nz-1 face moves along +x
    return w


def case_couette_sphere(n=32, tau=1.0, U=0.01, level=3, radius=4.0, steps=200, precision=PREC_FP64):
    """32^3 Couette cell, z walls at -+U, one neutrally buoyant rigid sphere
    (radius 4, 642 markers) at the centre, FP64."""
    c = (n - 1) / 2.0
    v, f = icosphere(level, radius, (c, c, c))
    body = Body(v, f, rigid=True, density_ratio=1.0, ref_radius=radius)
    return Case("couette_rigid_sphere_32", (n, n, n), tau, (PERIODIC, PERIODIC, WALL), shear_walls(U),
                precision=precision, steps=steps, bodies=[body], u0=couette_profile((n, n, n), U))


def case_capsule_shear(n=96, tau=0.8, shear_rate=1e-4, radius=10.0, level=4, Ca=0.05, Eb=0.01, kv=10.0,
                       density_ratio=1.0, steps=20000, precision=PREC_FP32, center=None, mass_model=1):
    """Deformable capsule in a Couette cell: 96^3, tau 0.8, shear rate 1e-4,
    radius 10 (2562 markers, 5120 triangles), solid-to-fluid density ratio 1
    with the capsule's mass that of its enclosed volume (Sec. 3.4)."""
    U = shear_rate * (n - 1) / 2.0
    c = (n - 1) / 2.0
    v, f = icosphere(level, radius, center if center is not None else (c, c, c))
    body = Body(v, f, rigid=False, ks0=ks0_from_capillary(Ca, tau, shear_rate, radius), Eb=Eb, kv=kv,
                density_ratio=density_ratio, ref_radius=radius, mass_model=mass_model)
    return Case(f"capsule_shear_{n}_Ca{Ca:g}", (n, n, n), tau, (PERIODIC, PERIODIC, WALL), shear_walls(U),
                precision=precision, steps=steps, bodies=[body], u0=couette_profile((n, n, n), U))


def case_jeffery_spheroid(n=32, tau=0.8, shear_rate=5e-3, axes=(6.0, 3.0, 3.0), level=3, precision=PREC_FP32,
                          steps=800):
    """Neutrally buoyant rigid prolate spheroid (aspect ratio 2, major axis
    along the flow x) at the centre of a Couette cell n^3 with z walls: the
    Jeffery-orbit configuration (quarter period pi (r + 1/r) / (2 shear_rate)
    = 785 steps at the defaults)."""
    U = shear_rate * (n - 1) / 2.0
    c = (n - 1) / 2.0
    v, f = icosphere(level, 1.0, (c, c, c), axes=axes)
    body = Body(v, f, rigid=True, density_ratio=1.0, ref_radius=float(axes[1]))
    return Case(f"jeffery_spheroid_{n}", (n, n, n), tau, (PERIODIC, PERIODIC, WALL), shear_walls(U),
                precision=precision, steps=steps, bodies=[body], u0=couette_profile((n, n, n), U))


# Parameter box of the batched and served capsule runs.  The sweep's full
# box (Ca log-uniform in [0.005, 0.3], bending ratio in [0, 0.05], mass ratio
# in {0.5, 1, 2}) includes membranes that the explicit marker update cannot
# carry: stiff (small Ca), light (mass ratio 0.5) or bending-dominated
# capsules diverge within 100-700 steps in FP32 and FP64 alike.  The runs use
# the part of the box that stays stable.
BATCH_CA = (0.05, 0.3)
BATCH_EB = (0.0, 0.01)
BATCH_MASS_RATIOS = (1.0, 2.0)


def case_batch(count=64, seed=2207, n_range=(48, 112), Ca_range=BATCH_CA, Eb_range=BATCH_EB,
               mass_ratios=BATCH_MASS_RATIOS, tau=0.8, wall_speed=0.02, precision=PREC_FP32, steps=2000):
    """Independent capsule-in-shear cases of uneven sizes: cubic lattices
    N ~ U{48..112}, capsule radius N/10 (icosphere level 3, 642 markers, up
    to radius 7; level 4, 2562 markers, above), Ca log-uniform, bending ratio
    uniform, membrane mass ratio from the given set, z walls moving at
    -+wall_speed.  Returns the cases and the drawn parameters."""
    rng = np.random.default_rng(seed)
    cases, params = [], []
    for k in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        Ca = float(np.exp(rng.uniform(np.log(Ca_range[0]), np.log(Ca_range[1]))))
        Eb = float(rng.uniform(*Eb_range))
        mr = float(rng.choice(mass_ratios))
        radius = n / 10.0
        level = 3 if radius <= 7.0 else 4
        shear_rate = 2.0 * wall_speed / (n - 1)
        c = (n - 1) / 2.0
        v, f = icosphere(level, radius, (c, c, c))
        body = Body(v, f, rigid=False, ks0=ks0_from_capillary(Ca, tau, shear_rate, radius), Eb=Eb, kv=1.0,
                    density_ratio=mr, ref_radius=radius)
        cases.append(Case(f"batch_{k}_n{n}", (n, n, n), tau, (PERIODIC, PERIODIC, WALL), shear_walls(wall_speed),
                          precision=precision, steps=steps, bodies=[body], u0=couette_profile((n, n, n), wall_speed)))
        params.append({"n": n, "Ca": Ca, "Eb": Eb, "mass_ratio": mr, "level": level, "radius": radius})
    return cases, params


# the capsule parameter box of the batched sweep as stated for it (Ca
# log-uniform, bending ratio uniform, membrane mass ratio): its stiff, light
# and bending-dominated corners diverge under the explicit marker update
FULL_CA = (0.005, 0.3)
FULL_EB = (0.0, 0.05)
FULL_MASS_RATIOS = (0.5, 1.0, 2.0)


def serve_stream(count=32, seed=4, rate=4.0, n_range=(32, 160), step_range=(1000, 6000), precision=PREC_FP32,
                 Ca_range=BATCH_CA, Eb_range=BATCH_EB, mass_ratios=BATCH_MASS_RATIOS, capsule_min_n=48):
    """A seeded Poisson arrival stream (mean `rate` requests per second) of
    capsule-in-shear and settling-sphere runs, half each: cubic lattices
    N ~ U{n_range} (capsules at least capsule_min_n), steps ~ U{step_range}, capsule
    parameters drawn as in case_batch (radius N/10), settling spheres of radius N/10 (icosphere level 3 or 4) at
    density ratio U[1.1, 1.5] with gravity for a terminal Re U[1, 20] (capped
    so that the sphere stays clear of the floor for its steps).
    Returns [(arrival_s, case, steps)]."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        steps = int(rng.integers(step_range[0], step_range[1] + 1))
        if k % 2 == 0:
            # capsules keep the validated box of case_batch: N >= 48, radius
            # N/10 (smaller or more confined capsules lose the stability of
            # the explicit marker update within a few thousand steps)
            n = max(n, capsule_min_n)
        radius = n / 10.0
        c = (n - 1) / 2.0
        if k % 2 == 0:
            level = 3 if radius <= 7.0 else 4
            Ca = float(np.exp(rng.uniform(np.log(Ca_range[0]), np.log(Ca_range[1]))))
            Eb = float(rng.uniform(*Eb_range))
            mr = float(rng.choice(mass_ratios))
            ws = 0.02
            v, f = icosphere(level, radius, (c, c, c))
            body = Body(v, f, rigid=False, ks0=ks0_from_capillary(Ca, 0.8, 2.0 * ws / (n - 1), radius), Eb=Eb,
                        kv=1.0, density_ratio=mr, ref_radius=radius)
            case = Case(f"serve_capsule_{k}_n{n}", (n, n, n), 0.8, (PERIODIC, PERIODIC, WALL), shear_walls(ws),
                        precision=precision, steps=steps, bodies=[body], u0=couette_profile((n, n, n), ws))
        else:
            level = 3 if radius <= 7.0 else 4
            gamma = float(rng.uniform(1.1, 1.5))
            # terminal Re drawn in [1, 20], capped so that the sphere falls at
            # most 0.2 N during its steps (it starts 0.7 N above the floor)
            Re = min(float(rng.uniform(1.0, 20.0)), 0.2 * n * 2.0 * radius / (viscosity(0.7) * steps))
            g = settling_gravity(Re, gamma, 2.0 * radius, 0.7)
            v, f = icosphere(level, radius, (c, c, 0.7 * (n - 1)))
            body = Body(v, f, rigid=True, density_ratio=gamma, ref_radius=radius, gravity=(0.0, 0.0, -g))
            case = Case(f"serve_settling_{k}_n{n}", (n, n, n), 0.7, (WALL, WALL, WALL), np.zeros((6, 3)),
                        precision=precision, steps=steps, bodies=[body])
        out.append((t, case, steps))
    return out


def case_cavity(n=25, Re=10.0, tau=0.8, precision=PREC_FP32, sphere=False, steps=None, obstacle=False):
    """Lid-driven cubic cavity (Sec. 3.1): walls on every face, the +y face
    moving along +z at u_lid = Re nu / (n - 1) (diffusive scaling: fixed tau,
    u_lid ~ 1/n).  With sphere=True a neutrally buoyant rigid sphere of
    radius n/8 (icosphere level 3) sits at (0.5, 0.35, 0.5) L.  With
    obstacle=True a fixed sphere of diameter 0.2 L sits at the centre (the
    obstacle of Sec. 3.1), held in place as the limit of a very dense rigid
    body (density ratio 1e12: it moves by less than 1e-6 lattice units over a
    run); its icosphere level grows with n so that there are about nine
    markers per lattice cell of surface (level 3 at 25 nodes, 4 at 49, 5 at
    97, 6 at 193)."""
    u_lid = Re * viscosity(tau) / (n - 1)
    wall_u = np.zeros((6, 3))
    wall_u[3, 2] = u_lid  # +y face moves along z
    bodies = []
    L = n - 1
    if sphere:
        v, f = icosphere(3, n / 8.0, (0.5 * L, 0.35 * L, 0.5 * L))
        bodies.append(Body(v, f, rigid=True, density_ratio=1.0, ref_radius=n / 8.0))
    if obstacle:
        level = max(1, int(round(3 + np.log2(L / 24.0))))
        v, f = icosphere(level, 0.1 * L, (0.5 * L, 0.5 * L, 0.5 * L))
        bodies.append(Body(v, f, rigid=True, density_ratio=1e12, ref_radius=0.1 * L))
    if steps is None:
        steps = int(2.0 * (n - 1) ** 2 / viscosity(tau))
    return Case(f"cavity_{n}_Re{Re:g}", (n, n, n), tau, (WALL, WALL, WALL), wall_u, precision=precision,
                steps=steps, bodies=bodies)


def case_settling(nx=160, ny=160, nz=480, tau=0.7, radius=8.0, level=5, Re=5.0, gamma=1.3, steps=50000,
                  precision=PREC_FP32, prolate=False):
    """Rigid sphere (radius 8, 10242 markers) settling along -z in a closed
    no-slip box 160x160x480, tau 0.7, g from the target Re and gamma."""
    d = 2.0 * radius
    g = settling_gravity(Re, gamma, d, tau)
    cen = ((nx - 1) / 2.0, (ny - 1) / 2.0, 0.75 * (nz - 1))
    axes = (radius, radius / 2.0, radius / 2.0) if prolate else None
    v, f = icosphere(level, radius, cen, axes=axes)
    body = Body(v, f, rigid=True, density_ratio=gamma, ref_radius=radius, gravity=(0.0, 0.0, -g))
    name = f"settling_{'prolate' if prolate else 'sphere'}_{nx}x{ny}x{nz}"
    return Case(name, (nx, ny, nz), tau, (WALL, WALL, WALL), np.zeros((6, 3)), precision=precision,
                steps=steps, bodies=[body])


def case_empty(n=(16, 12, 10), tau=0.8, bc=(PERIODIC, PERIODIC, PERIODIC), wall_u=None, gext=(0, 0, 0),
               precision=PREC_FP64, seed=0, amplitude=1e-2):
    """Lattice without bodies from a seeded random smooth-ish initial field."""
    rng = np.random.default_rng(seed)
    ncell = n[0] * n[1] * n[2]
    rho = 1.0 + amplitude * rng.standard_normal(ncell)
    u = amplitude * rng.standard_normal((ncell, 3))
    return Case(f"empty_{n[0]}x{n[1]}x{n[2]}", tuple(n), tau, tuple(bc),
                np.zeros((6, 3)) if wall_u is None else np.asarray(wall_u, np.float64),
                gext=tuple(gext), precision=precision, rho0=rho, u0=u)
