"""Batches (several contexts advanced by common launches) against the same
contexts stepped one by one, and against the FP64 oracle.

A batched context computes what lbib_step computes; only the order of the
atomic spreading sums may differ, so batched and alone agree to 1e-13
relative in FP64; in FP32 both are held to the FP32 bar against the oracle.
"""
import numpy as np
import pytest

import oracle
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


def mixed_cases(precision):
    """Uneven lattices: a capsule in shear, a settling sphere in a walled box,
    a body-free random periodic lattice, and two bodies (a membrane and a
    rigid sphere) in one lattice."""
    cases = [W.case_capsule_shear(n=30, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                  precision=precision)]
    v, f = W.icosphere(3, 3.5, (10.0, 11.0, 15.0))
    cases.append(W.Case("settle", (20, 22, 30), 0.7, (W.WALL, W.WALL, W.WALL), np.zeros((6, 3)), precision=precision,
                        bodies=[W.Body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.5,
                                       gravity=(0.0, 0.0, -2e-5))]))
    cases.append(W.case_empty(n=(18, 17, 19), precision=precision, seed=3))
    n = (34, 26, 27)
    U = 1e-3 * (n[2] - 1) / 2.0
    v1, f1 = W.icosphere(3, 5.0, (9.0, 12.0, 13.0))
    v2, f2 = W.icosphere(3, 3.0, (25.0, 13.0, 13.0))
    cases.append(W.Case("two", n, 0.8, (W.PERIODIC, W.PERIODIC, W.WALL), W.shear_walls(U), precision=precision,
                        u0=W.couette_profile(n, U),
                        bodies=[W.Body(v1, f1, rigid=False, ks0=W.ks0_from_capillary(0.05, 0.8, 1e-3, 5.0),
                                       Eb=0.01, kv=1.0, ref_radius=5.0),
                                W.Body(v2, f2, rigid=True, ref_radius=3.0)]))
    return cases


def state(ctx, case):
    return {"f": ctx.populations(), "u": ctx.fields()[1],
            "X": [ctx.markers(b)[0] for b in range(len(case.bodies))]}


def run_alone(L, cases, steps):
    out = []
    for case in cases:
        ctx = L.Context.from_case(case)
        ctx.step(steps)
        out.append(state(ctx, case))
        ctx.close()
    return out


@pytest.mark.parametrize("steps", [1, 13])
def test_fp64_batch_equals_contexts_alone(lbib, steps):
    cases = mixed_cases(W.PREC_FP64)
    alone = run_alone(lbib, cases, steps)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.step(steps)
    batch.sync()
    for ctx, case, a in zip(ctxs, cases, alone):
        s = state(ctx, case)
        assert rel(s["f"], a["f"]) < 1e-13
        assert rel(s["u"], a["u"]) < 1e-13
        for x, y in zip(s["X"], a["X"]):
            assert rel(x, y) < 1e-13
    nsteps, launches = batch.counters()
    assert nsteps == steps and launches >= steps
    batch.close()
    for ctx in ctxs:
        ctx.close()


def test_fp64_batch_matches_oracle(lbib):
    cases = mixed_cases(W.PREC_FP64)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.step(8)
    batch.step(5)
    for ctx, case in zip(ctxs, cases):
        s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
        s.set_fields(*case.initial_fields())
        for b in case.bodies:
            s.add_body(b.verts, b.tris, **b.kwargs())
        assert s.step(13) == 0
        assert rel(ctx.populations(), s.populations()) < 1e-12
        for k in range(len(case.bodies)):
            assert rel(ctx.markers(k)[0], s.markers(k)[0]) < 1e-12
        s.close()
    batch.close()
    for ctx in ctxs:
        ctx.close()


def oracle_state(case, steps):
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    for b in case.bodies:
        s.add_body(b.verts, b.tris, **b.kwargs())
    assert s.step(steps) == 0
    out = {"f": s.populations(), "u": s.fields()[1], "rho": s.fields()[0],
           "X": [s.markers(k)[0] for k in range(len(case.bodies))]}
    s.close()
    return out


def test_fp32_batch_matches_oracle_and_contexts_alone(lbib):
    """FP32 bar of the path: velocity within 1e-5 relative, density within
    1e-6, marker positions within 1e-4 lattice units of the oracle."""
    cases = mixed_cases(W.PREC_FP32)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.step(13)
    alone = run_alone(lbib, cases, 13)
    for ctx, case, a in zip(ctxs, cases, alone):
        s = state(ctx, case)
        o = oracle_state(case, 13)
        assert rel(s["u"], o["u"]) < 1e-5
        assert np.abs(ctx.fields()[0] - o["rho"]).max() < 1e-6
        for x, xo, xa in zip(s["X"], o["X"], a["X"]):
            assert np.abs(x - xo).max() < 1e-4
            assert np.abs(x - xa).max() < 1e-4
        assert rel(s["u"], a["u"]) < 1e-5
    batch.close()
    for ctx in ctxs:
        ctx.close()


def test_fp64_autotuned_batch_matches_oracle(lbib):
    """Every sweep block size and lattice order the batch autotuner tries
    computes the same steps: after tuning (which advances the runs) the
    state still matches the oracle advanced by as many steps."""
    cases = mixed_cases(W.PREC_FP64)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    threads, order, cpt = batch.autotune(1)
    assert threads in (0, 128, 256, 512) and order in (0, 1) and cpt in (1, 4)
    batch.step(3)
    taken = ctxs[0].counters()[0]
    for ctx, case in zip(ctxs, cases):
        assert ctx.counters()[0] == taken
        o = oracle_state(case, taken)
        assert rel(ctx.populations(), o["f"]) < 1e-12
        for k in range(len(case.bodies)):
            assert rel(ctx.markers(k)[0], o["X"][k]) < 1e-12
    batch.close()
    for ctx in ctxs:
        ctx.close()


def test_context_stepped_outside_the_batch_is_refused(lbib):
    cases = mixed_cases(W.PREC_FP32)[:2]
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.step(2)
    ctxs[1].step(1)
    with pytest.raises(lbib.LbibError) as ei:
        batch.step(1)
    assert ei.value.code == lbib.LBIB_EINVAL
    batch.close()
    batch = lbib.Batch(ctxs)  # rebuilt from the current state
    batch.step(3)
    batch.sync()
    batch.close()
    for ctx in ctxs:
        ctx.close()


@pytest.mark.parametrize("config", [(0, 1, 4), (128, 1, 1), (512, 0, 16), (64, 0, 3)])
def test_batch_configurations_compute_the_same_steps(lbib, config):
    """lbib_batch_set_config: per-lattice sweeps or the batched sweep in
    other shapes, FP64, against the contexts stepped alone."""
    cases = mixed_cases(W.PREC_FP64)
    alone = run_alone(lbib, cases, 8)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.set_config(*config)
    batch.step(8)
    batch.sync()
    for ctx, case, a in zip(ctxs, cases, alone):
        s = state(ctx, case)
        assert rel(s["f"], a["f"]) < 1e-13
        for x, y in zip(s["X"], a["X"]):
            assert rel(x, y) < 1e-13
    for bad in [(100, 0, 4), (1024, 0, 4), (256, 2, 4), (256, 0, 0), (256, 0, 17)]:
        with pytest.raises(lbib.LbibError) as ei:
            batch.set_config(*bad)
        assert ei.value.code == lbib.LBIB_EINVAL
    batch.close()
    for ctx in ctxs:
        ctx.close()


def test_batch_rejects_mixed_precisions(lbib):
    a = lbib.Context((8, 8, 8), 0.8, precision=lbib.LBIB_FP32)
    b = lbib.Context((8, 8, 8), 0.8, precision=lbib.LBIB_FP64)
    with pytest.raises(lbib.LbibError) as ei:
        lbib.Batch([a, b])
    assert ei.value.code == lbib.LBIB_EINVAL
    a.close()
    b.close()


def test_batch_with_centroid_marker_bodies_equals_contexts_alone(lbib):
    """Bodies with centroid IB markers (a capsule in shear, a settling sphere
    with the momentum-exchange force) batched with a vertex-marker body:
    the centroid spreading kernel of the batch computes what each context
    computes alone (FP64, 1e-13)."""
    cases = mixed_cases(W.PREC_FP64)[:3]
    cases[0].bodies[0].centroid_markers = 1
    cases[1].bodies[0].centroid_markers = 1
    cases[1].bodies[0].rigid_force = 1
    alone = run_alone(lbib, cases, 13)
    ctxs = [lbib.Context.from_case(c) for c in cases]
    batch = lbib.Batch(ctxs)
    batch.step(13)
    batch.sync()
    for ctx, case, a in zip(ctxs, cases, alone):
        st = state(ctx, case)
        assert rel(st["f"], a["f"]) < 1e-13
        for x, y in zip(st["X"], a["X"]):
            assert rel(x, y) < 1e-13
    batch.close()
    for ctx in ctxs:
        ctx.close()