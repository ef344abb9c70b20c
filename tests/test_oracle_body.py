"""Pins of the oracle's structure update and fluid-structure coupling (Sec. 2.3).

References: hand-computed integrator sequences, exactness of the backward
formulas on polynomials, Galilean invariance (a body moving with a uniform
flow feels no force), a stress-free membrane in a fluid at rest stays put,
the pressure-jump force of a linear density field (closed form), Stokes'
result that a neutrally buoyant sphere in simple shear spins at half the
shear rate, and the printed constants of Abraham's drag law.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2207_06029_gb300 import workloads as W


def test_verlet_hand_computed():
    """Eqs. (verletPos, verletVel), dt = 1."""
    # start-up (x(t-dt) = x(t)), U = 1, no force: tentative x = 1,
    # u = 1.5*1 - 2*0 + 0.5*0 = 1.5, x(t+dt) = 1.5
    xn, un = oracle.verlet([0, 0, 0], [0, 0, 0], [1, 0, 0], [0, 0, 0])
    assert np.array_equal(xn, [1.5, 0, 0]) and np.array_equal(un, [1.5, 0, 0])
    # uniform motion with the fluid is reproduced exactly
    xn, un = oracle.verlet([1, 2, 3], [0, 1, 2], [1, 1, 1], [0, 0, 0])
    assert np.array_equal(xn, [2, 3, 4]) and np.array_equal(un, [1, 1, 1])
    # constant acceleration a = 0.2, at rest: x~ = 0.1, u = 0.15, x = 0.25
    xn, un = oracle.verlet([0, 0, 0], [0, 0, 0], [0, 0, 0], [0.2, 0, 0])
    assert abs(xn[0] - 0.25) < 1e-16 and abs(un[0] - 0.15) < 1e-16


def test_bdf2_exact_for_linear_history():
    """Eqs. (linearVelRig, angularVelRig) reproduce v(t) = v0 + a t exactly."""
    v0, a = np.array([0.3, -0.1, 0.2]), np.array([0.01, 0.02, -0.03])
    for n in range(2, 6):
        out = oracle.bdf2(v0 + a * (n - 1), v0 + a * (n - 2), a)
        assert np.abs(out - (v0 + a * n)).max() < 1e-15


def test_rigid_body_galilean_invariance():
    """A rigid sphere translating with a uniform periodic flow: every probe
    sees the same state on both sides, the interpolated velocity equals the
    body's, and nothing changes except the translation."""
    n, U0 = 20, np.array([0.02, -0.01, 0.015])
    v, f = W.icosphere(2, 3.0, (9.7, 10.2, 9.9))
    s = oracle.Sim((n, n, n), 0.8)
    s.set_fields(np.ones(n ** 3), np.tile(U0, (n ** 3, 1)))
    s.add_body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.0, u0=tuple(U0))
    assert s.step(20) == 0
    rho, u = s.fields()
    assert np.abs(u - U0).max() < 1e-15 and np.abs(rho - 1).max() < 1e-14
    X, Ub, Fl = s.markers(0)
    assert np.abs(Fl).max() < 1e-15
    assert np.abs(X - (v + 20 * U0)).max() < 1e-12
    assert np.abs(s.body(0)["omega"]).max() < 1e-15


def test_membrane_at_rest_stays_at_rest():
    """Stress-free capsule in a fluid at rest: all forces vanish, so nothing
    moves beyond round-off."""
    n = 20
    v, f = W.icosphere(2, 4.0, (9.6, 9.4, 10.3))
    s = oracle.Sim((n, n, n), 0.7, bc=(0, 1, 0))
    # k_v = 1: the explicit update is stable for the collective radial mode
    # only while 1.25 * 3 k_v / (rho_s T r) < 2
    s.add_body(v, f, ks0=0.01, Eb=0.01, kv=1.0, ref_radius=4.0)
    assert s.step(15) == 0
    X, Ub, Fl = s.markers(0)
    assert np.abs(X - v).max() < 1e-13 and np.abs(Fl).max() < 1e-14
    rho, u = s.fields()
    assert np.abs(u).max() < 1e-14


def test_pressure_jump_of_linear_density(paper_const):
    """Eq. (hydroForP) on the field rho = 1 + beta.x, u = 0: the MLS fits are
    exact, p+ - p- = c_s^2 beta.(2 * 1.2 n), so
    F = -c_s^2 2.4 (beta.n) n A; Eq. (hydroForNu) adds nothing."""
    n = (16, 16, 16)
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    beta = np.array([1e-3, -2e-3, 5e-4])
    rho = (1.0 + beta[0] * x + beta[1] * y + beta[2] * z).ravel()
    u = np.zeros((rho.size, 3))
    v, f = W.icosphere(1, 3.0, (7.3, 7.9, 8.1))
    cs2, L = paper_const["cs2"], paper_const["probe_length"]
    for t in f[:10]:
        F = oracle.hydro_force_fields(n, (0, 0, 0), 0.1, rho, u, v, t)
        a, b, c = v[t[0]], v[t[1]], v[t[2]]
        N = np.cross(b - a, c - a)
        A = 0.5 * np.linalg.norm(N)
        nn = N / np.linalg.norm(N)
        ref = -cs2 * (2 * L) * (beta @ nn) * nn * A
        assert np.abs(F - ref).max() < 1e-15


def test_viscous_jump_vanishes_for_linear_flow():
    """A linear velocity field has the same stress on both probes."""
    n = (16, 16, 16)
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    G = np.array([[0.0, 1e-3, 2e-4], [3e-4, -1e-4, 0.0], [1e-4, 5e-4, 1e-4]])
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    u = pos @ G.T
    rho = np.ones(pos.shape[0])
    v, f = W.icosphere(1, 3.0, (7.3, 7.9, 8.1))
    for t in f[:10]:
        F = oracle.hydro_force_fields(n, (0, 0, 0), 0.1, rho, u, v, t)
        # round-off relative to the stress scale nu |G| A ~ 1e-4
        assert np.abs(F).max() < 1e-14


def test_neutral_sphere_spins_at_half_shear_rate():
    """Stokes: a free, neutrally buoyant sphere in simple shear rotates with
    omega = shear_rate/2 about the vorticity axis and stays at the centre.
    32^3 Couette cell, radius 4 (confinement a/H = 0.13), Re ~ 0.06."""
    case = W.case_couette_sphere(steps=200)
    s = oracle.Sim(case.n, case.tau, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    assert s.step(200) == 0
    st = s.body(0)
    gamma = 0.02 / 31.0
    assert abs(st["omega"][1] / (gamma / 2) - 1.0) < 0.02
    assert abs(st["omega"][0]) < 1e-12 and abs(st["omega"][2]) < 1e-12
    assert np.abs(st["xc"] - 15.5).max() < 1e-10


def test_settling_gravity_inverts_abraham_law(paper_const):
    """g from (Re, gamma) satisfies u_inf = sqrt(4 g d (gamma-1)/(3 C_d)) with
    C_d = C0 (1 + delta0/sqrt(Re))^2, C0 delta0^2 = 24, delta0 = 9.06."""
    d0 = paper_const["abraham_delta0"]
    C0 = paper_const["abraham_C0_delta0_sq"] / d0 ** 2
    for Re, gamma, d, tau in [(1.5, 1.14, 16, 0.7), (31.9, 1.16, 30, 0.6), (5, 1.3, 16, 0.7)]:
        g = W.settling_gravity(Re, gamma, d, tau)
        Cd = C0 * (1 + d0 / math.sqrt(Re)) ** 2
        u_inf = math.sqrt(4 * g * d * (gamma - 1) / (3 * Cd))
        assert abs(u_inf * d / ((tau - 0.5) / 3) - Re) < 1e-10 * Re


def test_support_reaching_a_wall_is_an_error():
    """A marker whose support touches a wall node stops the run with the
    body-wall error, and the error is sticky."""
    n = 16
    v, f = W.icosphere(1, 2.0, (8.0, 8.0, 3.2))
    s = oracle.Sim((n, n, n), 0.8, bc=(0, 0, 1))
    s.add_body(v, f, rigid=True, ref_radius=2.0)
    assert s.step(1) == oracle.EBODY_WALL
    assert s.step(1) == oracle.EBODY_WALL


def test_kinematic_membrane_is_carried_by_a_uniform_flow():
    """Kinematic IB (Sec. 3.4 variant): markers advected with the fluid.  A
    membrane at its rest shape feels no internal force, so in a uniform
    periodic flow it translates rigidly with the flow and leaves the fluid
    uniform (MLS reproduces the uniform field exactly)."""
    n = (20, 18, 22)
    u0 = np.array([0.01, -0.004, 0.002])
    v, f = W.icosphere(2, 3.5, (9.3, 8.1, 10.7))
    s = oracle.Sim(n, 0.8)
    ncell = n[0] * n[1] * n[2]
    s.set_fields(np.ones(ncell), np.tile(u0, (ncell, 1)))
    s.add_body(v, f, rigid=False, ks0=5e-3, Eb=0.01, kv=1.0, ref_radius=3.5, kinematic=1)
    assert s.step(10) == 0
    X = s.markers(0)[0]
    assert np.abs(X - (v + 10 * u0)).max() < 1e-12
    rho, u = s.fields()
    assert np.abs(u - u0).max() < 1e-13 and np.abs(rho - 1.0).max() < 1e-13
    s.close()


def test_momentum_exchange_sphere_spins_at_half_shear_rate():
    """The momentum-exchange rigid-body force (minus the IB force given to
    the fluid, plus the inertia of the enclosed fluid) gives the same Stokes
    rotation omega = shear_rate/2 of a free neutrally buoyant sphere as the
    printed stress-jump force (same 32^3 Couette cell, 200 steps)."""
    case = W.case_couette_sphere(steps=200)
    s = oracle.Sim(case.n, case.tau, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    kw = b.kwargs()
    kw["rigid_force"] = 1
    s.add_body(b.verts, b.tris, **kw)
    assert s.step(200) == 0
    st = s.body(0)
    gamma = 0.02 / 31.0
    assert abs(st["omega"][1] / (gamma / 2) - 1.0) < 0.02
    assert np.abs(st["xc"] - 15.5).max() < 1e-10
    s.close()


# ---------------------------------------------------------------------------------------
# centroid markers (the markers at the triangle centroids, as printed in Sec. 2.3)
# ---------------------------------------------------------------------------------------

def test_centroid_markers_rigid_galilean_invariance():
    """Centroid markers: a rigid sphere moving with a uniform periodic flow.
    MLS reproduces the uniform field at every centroid, the vertices'
    velocities (area-weighted means of their triangles') equal the flow's,
    and the body feels no force."""
    n, U0 = 20, np.array([0.02, -0.01, 0.015])
    v, f = W.icosphere(2, 3.0, (9.7, 10.2, 9.9))
    s = oracle.Sim((n, n, n), 0.8)
    s.set_fields(np.ones(n ** 3), np.tile(U0, (n ** 3, 1)))
    s.add_body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.0, u0=tuple(U0), centroid_markers=1)
    assert s.step(20) == 0
    rho, u = s.fields()
    assert np.abs(u - U0).max() < 1e-15 and np.abs(rho - 1).max() < 1e-14
    X, Ub, Fl = s.markers(0)
    assert np.abs(Fl).max() < 1e-15
    assert np.abs(X - (v + 20 * U0)).max() < 1e-12
    s.close()


def test_centroid_markers_kinematic_membrane_is_carried_by_a_uniform_flow():
    n = (20, 18, 22)
    u0 = np.array([0.01, -0.004, 0.002])
    v, f = W.icosphere(2, 3.5, (9.3, 8.1, 10.7))
    s = oracle.Sim(n, 0.8)
    ncell = n[0] * n[1] * n[2]
    s.set_fields(np.ones(ncell), np.tile(u0, (ncell, 1)))
    s.add_body(v, f, rigid=False, ks0=5e-3, Eb=0.01, kv=1.0, ref_radius=3.5, kinematic=1, centroid_markers=1)
    assert s.step(10) == 0
    assert np.abs(s.markers(0)[0] - (v + 10 * u0)).max() < 1e-12
    rho, u = s.fields()
    assert np.abs(u - u0).max() < 1e-13 and np.abs(rho - 1.0).max() < 1e-13
    s.close()


def vertex_areas(v, f):
    """A third of the area of each incident triangle (Sec. 2.3)."""
    A = 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
    Av = np.zeros(len(v))
    for q in range(3):
        np.add.at(Av, f[:, q], A / 3.0)
    return Av


@pytest.mark.parametrize("centroid", [0, 1])
def test_spread_force_total_is_the_membrane_force(centroid):
    """Momentum given to the fluid: the MLS weights sum to one at every
    marker, so the spread field totals sum_l c_l F_l.  With vertex markers
    (c_l = A_v, F_l = a_v the Newton acceleration) and with centroid markers
    (c_l = A_t, F_l the mean acceleration of the triangle's corners) both
    totals are sum_v A_v a_v.  A capsule in a sheared fluid with a density
    gradient (element stresses on every triangle), after one step."""
    n = 22
    v, f = W.icosphere(2, 4.0, (10.6, 11.2, 10.3))
    s = oracle.Sim((n, n, n), 0.8)
    idx = np.arange(n ** 3)
    cx, cz = idx % n, idx // (n * n)
    u = np.zeros((n ** 3, 3))
    u[:, 0] = 0.005 * (cz - 11.0) / 11.0
    s.set_fields(1.0 + 0.002 * (cx - 11.0), u)
    s.add_body(v, f, ks0=0.01, Eb=0.01, kv=1.0, ref_radius=4.0, centroid_markers=centroid)
    assert s.step(1) == 0
    Fl = s.markers(0)[2]
    want = (vertex_areas(v, f)[:, None] * Fl).sum(axis=0)
    got = s.fib().sum(axis=0)
    assert np.abs(want).max() > 1e-6
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    s.close()


@pytest.mark.parametrize("rigid_force", [0, 1])
def test_centroid_markers_sphere_spins_at_half_shear_rate(rigid_force):
    """Stokes' free neutrally buoyant sphere in shear with the IB markers at
    the centroids: omega = shear_rate/2, both rigid-body force readings."""
    case = W.case_couette_sphere(steps=200)
    s = oracle.Sim(case.n, case.tau, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    kw = b.kwargs()
    kw["centroid_markers"] = 1
    kw["rigid_force"] = rigid_force
    s.add_body(b.verts, b.tris, **kw)
    assert s.step(200) == 0
    st = s.body(0)
    gamma = 0.02 / 31.0
    assert abs(st["omega"][1] / (gamma / 2) - 1.0) < 0.02
    assert np.abs(st["xc"] - 15.5).max() < 1e-10
    s.close()


@pytest.mark.parametrize("centroid", [0, 1])
def test_kinematic_markers_take_the_linear_shear_velocity(centroid):
    """Couette flow started at f = f^eq(1, u) with u linear in z: the
    streamed moments of the first step are that linear field exactly (the
    D3Q19 moments cancel its quadratic terms) and MLS reproduces linear
    fields, so a kinematic membrane at its rest shape moves, in one step, by
    u at its vertices (vertex markers) or by the area-weighted mean of u at
    its triangles' centroids (centroid markers, c_l = A_t, a third to each
    corner)."""
    n = (24, 20, 25)
    U = 1e-3 * (n[2] - 1) / 2.0
    v, f = W.icosphere(2, 4.0, (11.3, 9.6, 12.2))
    s = oracle.Sim(n, 0.8, bc=(W.PERIODIC, W.PERIODIC, W.WALL), wall_u=W.shear_walls(U).ravel())
    s.set_fields(np.ones(n[0] * n[1] * n[2]), W.couette_profile(n, U))
    s.add_body(v, f, ks0=5e-3, Eb=0.01, kv=1.0, ref_radius=4.0, kinematic=1, centroid_markers=centroid)
    assert s.step(1) == 0

    def ux(z):
        return U * (2.0 * z / (n[2] - 1) - 1.0)

    if centroid:
        A = 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
        cz = v[f].mean(axis=1)[:, 2]
        num = np.zeros(len(v))
        for q in range(3):
            np.add.at(num, f[:, q], A / 3.0 * ux(cz))
        want_ux = num / vertex_areas(v, f)
    else:
        want_ux = ux(v[:, 2])
    d = s.markers(0)[0] - v
    assert np.abs(d[:, 0] - want_ux).max() < 1e-15
    assert np.abs(d[:, 1:]).max() < 1e-15
    if centroid:
        assert np.abs(want_ux - ux(v[:, 2])).max() > 1e-6  # the two readings differ
    s.close()
