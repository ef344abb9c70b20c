"""Serving: requests admitted by a memory budget and advanced together in a
continuously rebuilt batch return what each request computes alone.

Alone and in the mix differ only in the order of the atomic spreading sums:
FP64 results agree to 1e-13 relative.
"""
import time

import numpy as np
import pytest

from paper_2207_06029_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WAIT_S = 300.0


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


def requests(precision):
    """(case, steps): capsules in shear of three sizes and a settling sphere."""
    out = [(W.case_capsule_shear(n=30, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                 precision=precision), 40)]
    v, f = W.icosphere(3, 3.5, (10.0, 11.0, 15.0))
    out.append((W.Case("settle", (20, 22, 30), 0.7, (W.WALL, W.WALL, W.WALL), np.zeros((6, 3)),
                       precision=precision, bodies=[W.Body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.5,
                                                           gravity=(0.0, 0.0, -2e-5))]), 25))
    out.append((W.case_capsule_shear(n=36, tau=0.8, shear_rate=2e-3, radius=6.0, level=3, Ca=0.2, Eb=0.0, kv=1.0,
                                     precision=precision), 57))
    out.append((W.case_capsule_shear(n=26, tau=0.7, shear_rate=1e-3, radius=4.5, level=3, Ca=0.1, Eb=0.005,
                                     kv=1.0, precision=precision), 33))
    return out


def alone(L, case, steps):
    ctx = L.Context.from_case(case)
    ctx.step(steps)
    out = (ctx.populations(), [ctx.markers(b)[0] for b in range(len(case.bodies))])
    ctx.close()
    return out


def take(L, server, rid, case):
    rc, state = L.lbib_serve_wait(server, rid, WAIT_S)
    assert rc == L.LBIB_OK and state == L.LBIB_REQ_DONE, (rc, state)
    h, times, rc = L.lbib_serve_take(server, rid)
    assert rc == L.LBIB_OK and h is not None
    ctx = L.Context.adopt(h, case.n, [b.verts.shape[0] for b in case.bodies])
    out = (ctx.populations(), [ctx.markers(b)[0] for b in range(len(case.bodies))], ctx.counters()[0])
    ctx.close()
    return out, times


@pytest.mark.parametrize("batch_cells,order", [(0, 0), (40000, 0), (40000, 1)])
def test_each_result_is_the_same_alone_and_in_the_mix(lbib, batch_cells, order):
    """batch_cells = 0: every admitted run in every chunk; 40000: about one
    lattice per chunk, the runs with the least remaining work (order 0) or
    the earliest submitted (order 1), the others waiting resident."""
    reqs = requests(W.PREC_FP64)
    server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=16, max_active=8, batch_cells=batch_cells,
                                    batch_order=order)
    ids = []
    for k, (case, steps) in enumerate(reqs):
        ids.append(lbib.lbib_serve_submit(server, lbib.request_from_case(case, steps)))
        if k == 1:
            time.sleep(0.05)  # arrivals while earlier runs are on the GPU
    results = [take(lbib, server, rid, case) for rid, (case, _) in zip(ids, reqs)]
    stats = lbib.lbib_serve_stats(server)
    lbib.lbib_serve_destroy(server)
    assert stats["runs_done"] == len(reqs) and stats["runs_failed"] == 0
    assert stats["chunks"] >= 4
    for (case, steps), ((f, X, nsteps), times) in zip(reqs, results):
        assert nsteps == steps
        f0, X0 = alone(lbib, case, steps)
        assert rel(f, f0) < 1e-13
        for x, x0 in zip(X, X0):
            assert rel(x, x0) < 1e-13
        assert times["latency_s"] >= times["queued_s"] >= 0.0


def test_plain_mode_runs_one_at_a_time_in_arrival_order(lbib):
    reqs = requests(W.PREC_FP64)[:3]
    server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=10, max_active=8, mode=lbib.LBIB_SERVE_PLAIN)
    ids = [lbib.lbib_serve_submit(server, lbib.request_from_case(c, s)) for c, s in reqs]
    results = [take(lbib, server, rid, case) for rid, (case, _) in zip(ids, reqs)]
    lbib.lbib_serve_destroy(server)
    done = [t["done_s"] for _, t in results]
    assert done == sorted(done)
    for (case, steps), ((f, X, _), _) in zip(reqs, results):
        f0, X0 = alone(lbib, case, steps)
        assert rel(f, f0) < 1e-13


def test_memory_budget_limits_admission(lbib):
    reqs = requests(W.PREC_FP32)
    one = max(c.ncell for c, _ in reqs) * 300  # above any single run's estimate, below two of the larger
    server = lbib.lbib_serve_create(hbm_budget=one, chunk_steps=8, max_active=8)
    ids = [lbib.lbib_serve_submit(server, lbib.request_from_case(c, s)) for c, s in reqs]
    big = W.case_capsule_shear(n=64, radius=6.0, level=3, precision=W.PREC_FP32)
    too_big = lbib.lbib_serve_submit(server, lbib.request_from_case(big, 5))
    for rid, (case, _) in zip(ids, reqs):
        take(lbib, server, rid, case)
    rc, state = lbib.lbib_serve_wait(server, too_big, WAIT_S)
    assert rc == lbib.LBIB_ENOMEM and state == lbib.LBIB_REQ_FAILED
    stats = lbib.lbib_serve_stats(server)
    lbib.lbib_serve_destroy(server)
    assert stats["peak_bytes"] <= one
    assert stats["runs_done"] == len(reqs)


def test_taking_and_destroying_results_while_the_server_runs(lbib):
    """Results are taken and destroyed on the caller's thread while the
    worker keeps admitting, rebuilding and capturing batches: no run fails."""
    rng = np.random.default_rng(5)
    server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=20, max_active=16)
    ids, cases = [], []
    for k in range(14):
        n = int(rng.integers(24, 41))
        case = W.case_capsule_shear(n=n, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.1, Eb=0.005, kv=1.0,
                                    precision=W.PREC_FP32)
        ids.append(lbib.lbib_serve_submit(server, lbib.request_from_case(case, int(rng.integers(30, 90)))))
        cases.append(case)
        if k % 3 == 2:
            time.sleep(0.01)
    for rid in ids:
        rc, state = lbib.lbib_serve_wait(server, rid, WAIT_S)
        h, times, rc = lbib.lbib_serve_take(server, rid)
        assert rc == lbib.LBIB_OK, times["error"]
        lbib.lbib_destroy(h)
    stats = lbib.lbib_serve_stats(server)
    lbib.lbib_serve_destroy(server)
    assert stats["runs_done"] == len(ids) and stats["runs_failed"] == 0


def test_centroid_marker_runs_are_served_batched_and_plain(lbib):
    """A run whose capsule has centroid IB markers, served beside other runs
    in batched mode and alone in plain mode, returns what it computes
    alone."""
    reqs = requests(W.PREC_FP64)[:2]
    odd = W.case_capsule_shear(n=26, tau=0.7, shear_rate=1e-3, radius=4.5, level=3, Ca=0.1, Eb=0.005, kv=1.0,
                               precision=W.PREC_FP64)
    odd.bodies[0].centroid_markers = 1
    f0, X0 = alone(lbib, odd, 20)
    for mode in (lbib.LBIB_SERVE_BATCHED, lbib.LBIB_SERVE_PLAIN):
        server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=7, max_active=8, mode=mode)
        ids = [lbib.lbib_serve_submit(server, lbib.request_from_case(c, s)) for c, s in reqs]
        rid = lbib.lbib_serve_submit(server, lbib.request_from_case(odd, 20))
        (f, X, nsteps), _ = take(lbib, server, rid, odd)
        for i, (case, _) in zip(ids, reqs):
            take(lbib, server, i, case)
        stats = lbib.lbib_serve_stats(server)
        lbib.lbib_serve_destroy(server)
        assert stats["runs_done"] == 3 and stats["runs_failed"] == 0
        assert nsteps == 20 and rel(f, f0) < 1e-13 and rel(X[0], X0[0]) < 1e-13


def test_oldest_first_order_finishes_runs_in_submission_order(lbib):
    """With batch_cells below two lattices and the earliest submitted run
    first, the runs advance one at a time in submission order (the resident
    ones wait), so they finish in that order whatever their lengths; an
    unknown order is refused."""
    reqs = requests(W.PREC_FP32)
    server = lbib.lbib_serve_create(hbm_budget=8 << 30, chunk_steps=8, max_active=8, batch_cells=1,
                                    batch_order=lbib.LBIB_SERVE_OLDEST)
    ids = [lbib.lbib_serve_submit(server, lbib.request_from_case(c, s)) for c, s in reqs]
    results = [take(lbib, server, rid, case) for rid, (case, _) in zip(ids, reqs)]
    lbib.lbib_serve_destroy(server)
    done = [t["done_s"] for _, t in results]
    assert done == sorted(done)
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_serve_create(hbm_budget=8 << 30, batch_order=2)
    assert ei.value.code == lbib.LBIB_EINVAL
