"""Reduced-precision storage of the populations (FP16 and BF16 deviations
f_i - w_i, FP32 arithmetic; FP64 kept for the MLS solves, the volume and the
rigid-body update) against the FP64 oracle, on the two results the method
is run for (Sec. 3): the Taylor deformation D of a capsule in shear and the
Jeffery orbit of a rigid prolate spheroid.  Bar: within 1 % of the oracle.
FP32 storage is held to the same bar.

D is taken from the second-moment tensor M of the enclosed volume (the
equivalent ellipsoid has semi-axes sqrt(5 lambda_k / V)); the orbit by the
step at which the major axis passes the wall normal (a quarter period).
Both are diagnostics computed here from the returned markers / quaternion.
"""
import numpy as np
import pytest

import oracle
from paper_2207_06029_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06029_gb300 import build, lbib as L
    build.build()
    L.load()
    return L


def taylor_D(X, tris):
    """(L - B) / (L + B) of the ellipsoid with the mesh's volume second moments."""
    P = X - X.mean(axis=0)
    a, b, c = P[tris[:, 0]], P[tris[:, 1]], P[tris[:, 2]]
    v = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0  # signed tetrahedra with the centre
    s = a + b + c
    M = np.einsum("i,ij,ik->jk", v / 20.0, a, a) + np.einsum("i,ij,ik->jk", v / 20.0, b, b) \
        + np.einsum("i,ij,ik->jk", v / 20.0, c, c) + np.einsum("i,ij,ik->jk", v / 20.0, s, s)
    ax = np.sqrt(5.0 * np.linalg.eigvalsh(M) / v.sum())
    return (ax.max() - ax.min()) / (ax.max() + ax.min())


def test_taylor_D_of_an_ellipsoid():
    """The diagnostic itself: a scaled icosphere is a linear image of a mesh
    with isotropic second moments, so its D is exactly that of the ellipsoid
    with semi-axes (6, 4, 3): (6 - 3) / (6 + 3)."""
    v, f = W.icosphere(5, 1.0, (3.0, 2.0, 1.0), axes=(6.0, 4.0, 3.0))
    assert abs(taylor_D(v, f) - 1.0 / 3.0) < 1e-12


def major_axis_x(q):
    w, x, y, z = q
    return 1.0 - 2.0 * (y * y + z * z)  # x-component of the rotated body x axis


def quarter_period(samples):
    """Step at which the major axis' x component first changes sign (linear
    interpolation between samples)."""
    for (t0, d0), (t1, d1) in zip(samples, samples[1:]):
        if d0 > 0.0 >= d1:
            return t0 + (t1 - t0) * d0 / (d0 - d1)
    raise AssertionError("no quarter turn within the run")


CAPSULE = dict(n=36, tau=0.8, shear_rate=2e-3, radius=6.0, level=3, Ca=0.05, Eb=0.01, kv=1.0)
CAPSULE_STEPS = 600
JEFFERY_STEPS, JEFFERY_EVERY = 1000, 10


@pytest.fixture(scope="module")
def oracle_results():
    case = W.case_capsule_shear(precision=W.PREC_FP64, **CAPSULE)
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    assert s.step(CAPSULE_STEPS) == 0
    D = taylor_D(s.markers(0)[0], b.tris)
    s.close()
    case = W.case_jeffery_spheroid(precision=W.PREC_FP64)
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    samples = [(0, 1.0)]
    for k in range(JEFFERY_EVERY, JEFFERY_STEPS + 1, JEFFERY_EVERY):
        assert s.step(JEFFERY_EVERY) == 0
        samples.append((k, major_axis_x(s.body(0)["q"])))
    s.close()
    return {"D": D, "T4": quarter_period(samples)}


PRECISIONS = ["LBIB_FP32", "LBIB_FP16_DEV", "LBIB_BF16_DEV"]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_capsule_deformation_within_one_percent(lbib, oracle_results, prec):
    case = W.case_capsule_shear(precision=W.PREC_FP32, **CAPSULE)
    ctx = lbib.Context.from_case(case, precision=getattr(lbib, prec))
    ctx.step(CAPSULE_STEPS)
    D = taylor_D(ctx.markers(0)[0], case.bodies[0].tris)
    ctx.close()
    assert oracle_results["D"] > 0.2  # the capsule has deformed
    assert abs(D - oracle_results["D"]) <= 0.01 * oracle_results["D"], (D, oracle_results["D"])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_jeffery_quarter_period_within_one_percent(lbib, oracle_results, prec):
    case = W.case_jeffery_spheroid(precision=W.PREC_FP32)
    ctx = lbib.Context.from_case(case, precision=getattr(lbib, prec))
    samples = [(0, 1.0)]
    for k in range(JEFFERY_EVERY, JEFFERY_STEPS + 1, JEFFERY_EVERY):
        ctx.step(JEFFERY_EVERY)
        samples.append((k, major_axis_x(ctx.body(0)["q"])))
    ctx.close()
    T4 = quarter_period(samples)
    assert abs(T4 - oracle_results["T4"]) <= 0.01 * oracle_results["T4"], (T4, oracle_results["T4"])
