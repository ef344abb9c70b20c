"""Pins of the oracle's membrane network and geometry (Sec. 2.3).

References: forces are the negative gradient of the printed potentials
(central finite differences), internal forces carry no net force or moment,
everything vanishes in the stress-free shape, dihedral angles of Platonic
solids, exact mass properties of a cube, and icosphere convergence to the
sphere's area and volume.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2207_06029_gb300 import workloads as W


def _mesh(level=2, radius=3.0, seed=0, amp=0.08):
    v, f = W.icosphere(level, radius, (0.3, -0.2, 0.1))
    return W.perturb(v, amp, seed), v, f


def _rest(v, f, ks0=0.7, Eb=0.3, radius=3.0):
    h, ht = oracle.mesh_hinges(len(v), f)
    A = 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
    l0 = np.linalg.norm(v[h[:, 0]] - v[h[:, 1]], axis=1)
    ks = ks0 * (A[ht[:, 0]] + A[ht[:, 1]]) / l0 ** 2
    th0 = np.array([oracle.hinge_theta(v[a], v[b], v[c], v[d]) for a, b, c, d in h])
    return h, ks, l0, Eb * ks * radius ** 2, th0


def _fd_check(energy, X, F, rng, ncheck=40, h=1e-6, rtol=1e-6):
    idx = rng.choice(X.size, size=ncheck, replace=False)
    Xf = X.ravel()
    scale = np.abs(F).max()
    for j in idx:
        Xp, Xm = Xf.copy(), Xf.copy()
        Xp[j] += h
        Xm[j] -= h
        g = (energy(Xp.reshape(X.shape)) - energy(Xm.reshape(X.shape))) / (2 * h)
        assert abs(-g - F.ravel()[j]) <= rtol * scale + 1e-12, (j, -g, F.ravel()[j])


def test_icosphere_counts_and_orientation():
    for L in range(4):
        v, f = W.icosphere(L, 1.0)
        assert len(v) == 10 * 4 ** L + 2 and len(f) == 20 * 4 ** L
        assert oracle.volume(v, f) > 0
        h, _ = oracle.mesh_hinges(len(v), f)
        assert len(h) == 30 * 4 ** L


def test_icosphere_converges_to_sphere():
    r = 2.5
    errs = []
    for L in range(1, 6):
        v, f = W.icosphere(L, r)
        errs.append((abs(oracle.volume(v, f) - 4 / 3 * math.pi * r ** 3) / (4 / 3 * math.pi * r ** 3),
                     abs(oracle.area(v, f) - 4 * math.pi * r ** 2) / (4 * math.pi * r ** 2)))
    errs = np.array(errs)
    assert np.all(np.diff(errs, axis=0) < 0)
    assert errs[-1, 0] < 2e-3 and errs[-1, 1] < 2e-3


def test_cube_mass_properties():
    """Unit-density cube of side a: V = a^3, centroid at its centre,
    I = a^5/6 on the diagonal (closed form)."""
    a = 1.7
    v, f = W.cube_mesh(a, center=(0.3, -1.1, 2.0))
    V, c, I = oracle.mass_properties(v, f)
    assert abs(V - a ** 3) < 1e-14
    assert np.abs(c - [0.3, -1.1, 2.0]).max() < 1e-14
    assert np.abs(I - a ** 5 / 6 * np.eye(3)).max() < 1e-13


def test_sphere_inertia_approaches_closed_form():
    r = 2.0
    v, f = W.icosphere(5, r)
    V, c, I = oracle.mass_properties(v, f)
    assert np.abs(c).max() < 1e-12
    Iref = 0.4 * V * r ** 2
    assert np.abs(I - Iref * np.eye(3)).max() / Iref < 5e-3


def test_dihedral_of_platonic_solids():
    """theta is the angle between the outward normals of the two triangles of
    a hinge, i.e. pi minus the interior dihedral angle: arccos(sqrt(5)/3) on
    an icosahedron (interior angle arccos(-sqrt(5)/3)), pi - arccos(1/3) on a
    regular tetrahedron, pi/2 across a cube's edges (0 on face diagonals)."""
    v, f = W.icosphere(0, 1.0)
    h, _ = oracle.mesh_hinges(len(v), f)
    th = [oracle.hinge_theta(*v[list(q)]) for q in h]
    assert np.abs(np.array(th) - math.acos(math.sqrt(5) / 3)).max() < 1e-14
    t = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    tf = W._orient_outward(t, np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]])).astype(np.int32)
    h, _ = oracle.mesh_hinges(4, tf)
    th = [oracle.hinge_theta(*t[list(q)]) for q in h]
    assert np.abs(np.array(th) - (math.pi - math.acos(1 / 3))).max() < 1e-14
    cv, cf = W.cube_mesh(1.0)
    h, _ = oracle.mesh_hinges(len(cv), cf)
    th = np.sort(np.abs([oracle.hinge_theta(*cv[list(q)]) for q in h]))
    assert np.abs(th[:6]).max() < 1e-15 and np.abs(th[6:] - math.pi / 2).max() < 1e-15


def test_dihedral_sign_convex_positive_and_gradient():
    rng = np.random.default_rng(2)
    for _ in range(30):
        xa, xb, xc, xd = rng.standard_normal((4, 3))
        th, g = oracle.hinge_theta(xa, xb, xc, xd, with_grad=True)
        assert np.abs(g.sum(0)).max() < 1e-12
        P = np.stack([xa, xb, xc, xd])
        for q in range(4):
            for k in range(3):
                Pp, Pm = P.copy(), P.copy()
                Pp[q, k] += 1e-7
                Pm[q, k] -= 1e-7
                fd = (oracle.hinge_theta(*Pp) - oracle.hinge_theta(*Pm)) / 2e-7
                assert abs(fd - g[q, k]) < 1e-6 * max(1, abs(g[q, k]))
    v, f = W.icosphere(2, 1.0)
    h, _ = oracle.mesh_hinges(len(v), f)
    assert min(oracle.hinge_theta(*v[list(q)]) for q in h) > 0


def test_spring_forces_are_energy_gradient():
    rng = np.random.default_rng(4)
    X, v, f = _mesh()
    h, ks, l0, _, _ = _rest(v, f)
    edges = h[:, :2].copy()
    E, F = oracle.spring_forces(X, edges, ks, l0)
    _fd_check(lambda Y: oracle.spring_forces(Y, edges, ks, l0)[0], X, F, rng)
    assert np.abs(F.sum(0)).max() < 1e-12
    assert np.abs(np.cross(X, F).sum(0)).max() < 1e-11
    E0, F0 = oracle.spring_forces(v, edges, ks, l0)
    assert E0 == 0.0 and np.abs(F0).max() == 0.0


@pytest.mark.parametrize("variant", [0, 1])
def test_bending_forces_are_energy_gradient(variant):
    rng = np.random.default_rng(5 + variant)
    X, v, f = _mesh(seed=3)
    h, _, _, kb, th0 = _rest(v, f)
    E, F = oracle.bend_forces(X, h, kb, th0, variant)
    _fd_check(lambda Y: oracle.bend_forces(Y, h, kb, th0, variant)[0], X, F, rng)
    assert np.abs(F.sum(0)).max() < 1e-11
    assert np.abs(np.cross(X, F).sum(0)).max() < 1e-10
    E0, F0 = oracle.bend_forces(v, h, kb, th0, variant)
    assert E0 == 0.0 and np.abs(F0).max() < 1e-15


def test_bending_variants_agree_to_second_order():
    """k_b [1 - cos d] = 1/2 k_b d^2 + O(d^4)."""
    X, v, f = _mesh(seed=8, amp=1e-3)
    h, _, _, kb, th0 = _rest(v, f)
    E0, F0 = oracle.bend_forces(X, h, kb, th0, 0)
    E1, F1 = oracle.bend_forces(X, h, kb, th0, 1)
    assert abs(E0 - E1) < 1e-3 * E1
    assert np.abs(F0 - F1).max() < 1e-3 * np.abs(F1).max()


def test_volume_forces_are_energy_gradient():
    rng = np.random.default_rng(6)
    X, v, f = _mesh(seed=4)
    V0 = oracle.volume(v, f)
    E, F = oracle.volume_forces(X, f, 10.0, V0)
    _fd_check(lambda Y: oracle.volume_forces(Y, f, 10.0, V0)[0], X, F, rng)
    assert np.abs(F.sum(0)).max() < 1e-12
    assert np.abs(np.cross(X, F).sum(0)).max() < 1e-11
    # restoring: a compressed capsule is pushed outward
    Xs = 0.97 * (v - v.mean(0)) + v.mean(0)
    _, Fs = oracle.volume_forces(Xs, f, 10.0, V0)
    assert np.all(np.einsum("ij,ij->i", Fs, Xs - Xs.mean(0)) > 0)


def test_rest_membrane_parameters(paper_const):
    """Van Gelder spring constants k_{s,l} = k_s0 T (A1 + A2)/l0^2, bending
    constant k_b = Eb k_{s,l} r^2 and vertex mass from the rest mesh."""
    v, f = W.icosphere(2, 3.0, (10, 10, 10))
    s = oracle.Sim((24, 24, 24), 0.8)
    s.add_body(v, f, ks0=0.02, Eb=0.01, kv=paper_const["capsule_kv"], thickness=1.0, density_ratio=2.0,
               ref_radius=3.0)
    r = s.body_rest(0)
    h, ks, l0, kb, th0 = _rest(v, f, ks0=0.02, Eb=0.01, radius=3.0)
    assert np.array_equal(r["hinge"], h)
    assert np.abs(r["ks"] - ks).max() < 1e-15 and np.abs(r["l0"] - l0).max() < 1e-15
    assert np.abs(r["kb"] - kb).max() < 1e-15
    assert abs(r["mv"] - 2.0 * oracle.area(v, f) / len(v)) < 1e-14


@pytest.mark.parametrize("radius,level", [(4.0, 3), (10.0, 4)])
def test_capsule_mass_model_is_that_of_the_enclosed_volume(radius, level):
    """Sec. 3.4 defines the capsule's mass by a solid-to-fluid density ratio:
    with mass_model 1 the vertices share rho_s V0 (V0 the enclosed volume),
    with mass_model 0 (the shell of unit thickness of Sec. 3.5) rho_s T A0.
    For a sphere the ratio of the two is V0 / (T A0) -> r / 3 as the mesh is
    refined (exact for the sphere's volume and area)."""
    v, f = W.icosphere(level, radius, (16.0, 16.0, 16.0))
    masses = {}
    for model in (0, 1):
        s = oracle.Sim((34, 34, 34), 0.8)
        s.add_body(v, f, ks0=0.01, Eb=0.0, kv=1.0, thickness=1.0, density_ratio=1.5, ref_radius=radius,
                   mass_model=model)
        masses[model] = s.body_rest(0)["mv"] * len(v)
        s.close()
    assert abs(masses[0] - 1.5 * oracle.area(v, f)) < 1e-12 * masses[0]
    assert abs(masses[1] - 1.5 * oracle.volume(v, f)) < 1e-12 * masses[1]
    sphere = (4.0 / 3.0 * np.pi * radius ** 3) / (4.0 * np.pi * radius ** 2)
    assert abs(masses[1] / masses[0] / sphere - 1.0) < 0.03
