"""Divergence detection: runs outside the scheme's stability range fail with
LBIB_EDIVERGED instead of finishing on NaNs, and a diverged run in the
serving mix fails alone while the others return what they compute alone.

The unstable cases diverge through plain floating-point arithmetic (values
grow, then overflow to inf or NaN); every index the kernels form from such
values is clamped or wrapped, and the marker coordinates are checked before
any node index is formed from them.
"""
import numpy as np
import pytest

from paper_2207_06029_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06029_gb300 import build, lbib as L
    build.build()
    L.load()
    return L


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def unstable_capsule(precision):
    """The stiff, light, bending-dominated corner of the batched capsule
    parameter box (N 48, Ca 0.005, Eb 0.05, mass ratio 0.5, walls at -+0.02):
    the explicit marker update amplifies the membrane's stiffest mode by an
    order of magnitude per step (the FP64 oracle moves a vertex by 0.12
    lattice units in step 4 and by 2.9 in step 5)."""
    n, tau, wall = 48, 0.8, 0.02
    rate = 2 * wall / (n - 1)
    radius = n / 10.0
    c = (n - 1) / 2.0
    v, f = W.icosphere(3, radius, (c, c, c))
    body = W.Body(v, f, rigid=False, ks0=W.ks0_from_capillary(0.005, tau, rate, radius), Eb=0.05, kv=1.0,
                  density_ratio=0.5, ref_radius=radius)
    return W.Case("capsule_unstable_48", (n, n, n), tau, (W.PERIODIC, W.PERIODIC, W.WALL), W.shear_walls(wall),
                  precision=precision, bodies=[body], u0=W.couette_profile((n, n, n), wall))


def shear_waves(n=16, amp=0.35):
    """Periodic n^3 fluid with two crossed sine shear waves of amplitude amp:
    at tau 0.5002 (viscosity 7e-5) the BGK scheme leaves its range, a node
    passing the speed of sound near step 25 (FP64 oracle)."""
    x = np.arange(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((n, n, n, 3))
    u[..., 0] = amp * np.sin(2 * np.pi * Y / n)
    u[..., 1] = amp * np.sin(2 * np.pi * Z / n)
    return np.ones(n ** 3), np.ascontiguousarray(u.transpose(2, 1, 0, 3).reshape(-1, 3))


def test_unstable_membrane_fails_with_ediverged(lbib):
    case = unstable_capsule(W.PREC_FP32)
    ctx = lbib.Context.from_case(case)
    ctx.step(30)
    with pytest.raises(lbib.LbibError) as ei:
        ctx.sync()
    assert ei.value.code == lbib.LBIB_EDIVERGED
    assert "diverged" in str(ei.value)
    # sticky: further steps are refused with the same code
    with pytest.raises(lbib.LbibError) as ei:
        ctx.step(1)
    assert ei.value.code == lbib.LBIB_EDIVERGED
    ctx.close()


def test_fluid_watchdog_flags_a_supersonic_run_only_when_on(lbib):
    rho, u = shear_waves()
    out = {}
    for every in (0, 10):
        ctx = lbib.Context((16, 16, 16), 0.5002, precision=lbib.LBIB_FP32)
        ctx.set_fields(rho, u)
        lbib.lbib_set_watchdog(ctx.h, every)
        ctx.step(40)
        try:
            ctx.sync()
            out[every] = lbib.LBIB_OK
        except lbib.LbibError as e:
            out[every] = e.code
        if every == 0:
            # the on-demand check sees it too
            with pytest.raises(lbib.LbibError) as ei:
                lbib.lbib_check(ctx.h)
            assert ei.value.code == lbib.LBIB_EDIVERGED
        ctx.close()
    assert out == {0: lbib.LBIB_OK, 10: lbib.LBIB_EDIVERGED}


def test_mass_drift_beyond_the_tolerance(lbib):
    """A piston: the -z wall moves into the box (Zou-He inflow), the +z wall
    is at rest, so mass enters at ~0.01 * 144 per step (0.06 % of the box a
    step): a 1e-3 tolerance trips within 20 steps, 0.5 does not; with the
    walls moving tangentially mass stays within 1e-12."""
    n = (12, 12, 16)
    for wall_u, tol, expect in [((0.0, 0.0, 0.01), 1e-3, "diverged"), ((0.0, 0.0, 0.01), 0.5, "ok"),
                                ((0.01, 0.0, 0.0), 1e-12, "ok")]:
        w = np.zeros((6, 3))
        w[4] = wall_u
        ctx = lbib.Context(n, 0.8, bc=(0, 0, 1), wall_u=w, precision=lbib.LBIB_FP64)
        lbib.lbib_set_watchdog(ctx.h, 10, tol)
        ctx.step(20)
        if expect == "ok":
            ctx.sync()
            assert lbib.lbib_check(ctx.h) == lbib.LBIB_OK
        else:
            with pytest.raises(lbib.LbibError) as ei:
                ctx.sync()
            assert ei.value.code == lbib.LBIB_EDIVERGED
        ctx.close()


def test_watchdog_leaves_the_run_unchanged(lbib):
    """A stable FP64 capsule run with the watchdog after every step and with
    it off: the same populations and markers (1e-13: only the order of the
    atomic spreading sums differs between two runs)."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    out = []
    for every in (1, 0):
        ctx = lbib.Context.from_case(case)
        lbib.lbib_set_watchdog(ctx.h, every)
        ctx.step(25)
        out.append((ctx.populations(), ctx.markers(0)[0]))
        ctx.close()
    assert rel(out[0][0], out[1][0]) < 1e-13 and rel(out[0][1], out[1][1]) < 1e-13


def test_serving_fails_the_diverged_run_alone(lbib):
    """Three stable FP64 runs and the unstable capsule submitted together
    (all admitted into one batch): the unstable run fails with
    LBIB_EDIVERGED, each stable run returns what it computes alone (1e-13:
    only the order of the atomic spreading sums differs)."""
    stable = [(W.case_capsule_shear(n=30, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                    kv=1.0, precision=W.PREC_FP64), 40),
              (W.case_capsule_shear(n=36, tau=0.8, shear_rate=2e-3, radius=6.0, level=3, Ca=0.2, Eb=0.0, kv=1.0,
                                    precision=W.PREC_FP64), 57),
              (W.case_capsule_shear(n=26, tau=0.7, shear_rate=1e-3, radius=4.5, level=3, Ca=0.1, Eb=0.005,
                                    kv=1.0, precision=W.PREC_FP64), 33)]
    ref = []
    for case, steps in stable:
        ctx = lbib.Context.from_case(case)
        ctx.step(steps)
        ref.append((ctx.populations(), ctx.markers(0)[0]))
        ctx.close()
    server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=16, max_active=8)
    bad = unstable_capsule(W.PREC_FP64)
    ids = [lbib.lbib_serve_submit(server, lbib.request_from_case(case, steps)) for case, steps in stable[:2]]
    bad_id = lbib.lbib_serve_submit(server, lbib.request_from_case(bad, 60))
    ids.append(lbib.lbib_serve_submit(server, lbib.request_from_case(*stable[2])))
    rc, state = lbib.lbib_serve_wait(server, bad_id, 300.0)
    assert rc == lbib.LBIB_EDIVERGED and state == lbib.LBIB_REQ_FAILED
    h, times, rc = lbib.lbib_serve_take(server, bad_id)
    assert rc == lbib.LBIB_EDIVERGED and h is None and "diverged" in times["error"]
    for rid, (case, steps), (f_ref, X_ref) in zip(ids, stable, ref):
        rc, state = lbib.lbib_serve_wait(server, rid, 300.0)
        assert rc == lbib.LBIB_OK and state == lbib.LBIB_REQ_DONE, (rc, state)
        h, times, rc = lbib.lbib_serve_take(server, rid)
        ctx = lbib.Context.adopt(h, case.n, [b.verts.shape[0] for b in case.bodies])
        assert ctx.counters()[0] == steps
        assert rel(ctx.populations(), f_ref) < 1e-13
        assert rel(ctx.markers(0)[0], X_ref) < 1e-13
        ctx.close()
    stats = lbib.lbib_serve_stats(server)
    assert stats["runs_failed"] == 1 and stats["runs_done"] == 3
    lbib.lbib_serve_destroy(server)
