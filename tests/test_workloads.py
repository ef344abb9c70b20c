"""The synthetic cases (host logic, no GPU): the geometry and parameters
the parity tests, the physics studies and the benchmark are built from."""
import numpy as np

from paper_2207_06029_gb300 import workloads as W


def test_shear_walls_and_couette_profile():
    """z walls moving along -x and +x at U; the profile is linear in z,
    -U and +U on the wall nodes, zero in y and z."""
    U, n = 0.01, (5, 4, 11)
    w = W.shear_walls(U)
    assert w[4, 0] == -U and w[5, 0] == U and np.count_nonzero(w) == 2
    u = W.couette_profile(n, U).reshape(n[2], n[1], n[0], 3)
    assert np.allclose(u[0, ..., 0], -U) and np.allclose(u[-1, ..., 0], U)
    assert np.allclose(np.diff(u[:, 0, 0, 0]), 2 * U / (n[2] - 1))
    assert not np.any(u[..., 1:])


def test_cavity_lid_and_fixed_obstacle():
    """The +y face moves along +z at Re nu / (n - 1); the obstacle of
    Sec. 3.1 is a sphere of diameter 0.2 L at the centre, its icosphere
    level growing with n (about nine markers per cell of surface), held in
    place as a very dense rigid body."""
    for n, level in ((25, 3), (49, 4), (97, 5)):
        c = W.case_cavity(n=n, Re=10.0, tau=0.8, obstacle=True)
        L = n - 1
        assert c.wall_u[3, 2] == 10.0 * W.viscosity(0.8) / L and np.count_nonzero(c.wall_u) == 1
        assert c.bc == (W.WALL, W.WALL, W.WALL)
        b = c.bodies[0]
        assert b.rigid and b.density_ratio >= 1e12
        assert len(b.verts) == 10 * 4 ** level + 2
        r = np.linalg.norm(b.verts - 0.5 * L, axis=1)
        assert np.allclose(r, 0.1 * L)
        per_cell = len(b.verts) / (4 * np.pi * (0.1 * L) ** 2)
        assert 8.0 < per_cell < 10.0


def test_capsule_case_uses_the_capsule_mass():
    """The capsule in shear of Sec. 3.4 carries the mass of its enclosed
    volume at the given density ratio (mass model 1); the batched and
    served capsules keep the shell model (0)."""
    c = W.case_capsule_shear(n=32, radius=5.0, level=2)
    assert c.bodies[0].mass_model == 1 and not c.bodies[0].rigid
    cases, _ = W.case_batch(count=4)
    assert all(b.mass_model == 0 for case in cases for b in case.bodies)
