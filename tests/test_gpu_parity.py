"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances: the FP64 build agrees with the oracle to 1e-12 relative
(populations, fields, markers); the FP32 build to 1e-5 relative on the
velocity field and 1e-4 lattice units on marker positions.  Relative means
max |gpu - oracle| / max |oracle| over the array.
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


def run_gpu(L, case, steps, precision=None):
    ctx = L.Context.from_case(case, precision=precision)
    ctx.step(steps)
    out = {"f": ctx.populations() if case.ncell <= 4_000_000 else None, "fields": ctx.fields(),
           "markers": [ctx.markers(b) for b in range(len(case.bodies))],
           "bodies": [ctx.body(b) for b in range(len(case.bodies))]}
    ctx.close()
    return out


def run_oracle(case, steps):
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    for b in case.bodies:
        s.add_body(b.verts, b.tris, **b.kwargs())
    rc = s.step(steps)
    assert rc == 0
    out = {"f": s.populations() if case.ncell <= 4_000_000 else None, "fields": s.fields(),
           "markers": [s.markers(b) for b in range(len(case.bodies))],
           "bodies": [s.body(b) for b in range(len(case.bodies))]}
    s.close()
    return out


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def check_fp64(g, o, tol=1e-12):
    """Populations, density and marker positions within tol relative; the
    velocity field within tol of max(|u|, 1e-2): a velocity far below the
    wall speeds is a cancellation of O(0.1) populations, so its rounding is
    absolute.  The marker boundary velocity U_b and the IB force F_l = U_b - U
    are held to tol of the velocity scale they are formed from (the larger of
    the flow's speed and 1e-2): F_l is a difference of nearly equal
    velocities, so its own size is no scale for its rounding."""
    if o["f"] is not None:
        assert rel(g["f"], o["f"]) < tol
    assert rel(g["fields"][0], o["fields"][0]) < tol
    uo = o["fields"][1]
    uscale = max(np.abs(uo).max(), 1e-2)
    assert np.abs(g["fields"][1] - uo).max() < tol * uscale
    for (Xg, Vg, Fg), (Xo, Vo, Fo) in zip(g["markers"], o["markers"]):
        assert rel(Xg, Xo) < tol
        vscale = max(uscale, np.abs(Vo).max())
        assert np.abs(Vg - Vo).max() < tol * vscale
        assert np.abs(Fg - Fo).max() < tol * vscale


# ---------------------------------------------------------------------------------------
# FP64: the fluid alone
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [(3, 4, 5), (33, 17, 9)])
def test_fp64_periodic_random_state(lbib, n):
    """Tiny and ragged periodic lattices from a random populated state, with a
    uniform body force (pull streaming and wrap at every face)."""
    case = W.case_empty(n=n, tau=0.73, gext=(1e-5, -2e-5, 3e-6), seed=1)
    rng = np.random.default_rng(2)
    e, w = oracle.lattice()
    f0 = w[None, :] * (1.0 + 0.02 * rng.standard_normal((case.ncell, 19)))
    ctx = lbib.Context(case.n, case.tau, body_force=case.gext, precision=lbib.LBIB_FP64)
    ctx.set_populations(f0)
    ctx.step(7)
    fg = ctx.populations()
    rg, ug = ctx.fields()
    ctx.close()
    s = oracle.Sim(case.n, case.tau, gext=case.gext)
    s.set_populations(f0.ravel())
    assert s.step(7) == 0
    assert rel(fg, s.populations()) < 1e-12
    ro, uo = s.fields()
    assert rel(rg, ro) < 1e-12 and rel(ug, uo) < 1e-12


@pytest.mark.parametrize("bc", [(1, 1, 1), (0, 1, 1), (1, 0, 0)])
def test_fp64_moving_walls_edges_corners(lbib, bc):
    """Walled boxes with tangentially moving walls: Zou-He faces plus the
    edge and corner rule."""
    n = (7, 6, 9)
    rng = np.random.default_rng(3)
    wall_u = 0.02 * rng.standard_normal((6, 3))
    for f in range(6):
        wall_u[f, f // 2] = 0.0  # tangential wall motion
    case = W.case_empty(n=n, tau=0.9, bc=bc, wall_u=wall_u, seed=4, amplitude=5e-3)
    g = run_gpu(lbib, case, 25, precision=lbib.LBIB_FP64)
    o = run_oracle(case, 25)
    check_fp64(g, o)


# ---------------------------------------------------------------------------------------
# FP64: immersed bodies
# ---------------------------------------------------------------------------------------

def test_fp64_couette_rigid_sphere_full(lbib):
    """32^3 Couette cell, z walls at -+0.01, rigid neutrally buoyant sphere of
    radius 4 (642 markers), tau 1, 200 steps, FP64."""
    case = W.case_couette_sphere()
    g = run_gpu(lbib, case, case.steps)
    o = run_oracle(case, case.steps)
    check_fp64(g, o)
    bg, bo = g["bodies"][0], o["bodies"][0]
    assert np.abs(bg["omega"] - bo["omega"]).max() < 1e-12 * np.abs(bo["omega"]).max()
    assert np.abs(bg["xc"] - bo["xc"]).max() < 1e-12 * 16


@pytest.mark.parametrize("bend_variant", [0, 1])
def test_fp64_capsule_in_shear(lbib, bend_variant):
    """Deformable capsule (springs, bending, volume, probes, Verlet) in a 24^3
    Couette cell, 40 steps, FP64."""
    # Eb = 0.01 keeps the explicit update stable at this resolution (0.05
    # diverges in the oracle as well)
    case = W.case_capsule_shear(n=24, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    case.bodies[0].bend_variant = bend_variant
    case.bodies[0].verts = W.perturb(case.bodies[0].verts, 0.02, seed=11)
    g = run_gpu(lbib, case, 40)
    o = run_oracle(case, 40)
    check_fp64(g, o)


def test_fp64_kinematic_capsule_in_shear(lbib):
    """Kinematic-IB variant (markers advected with the interpolated fluid
    velocity, internal forces spread), 28^3, 25 steps."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    case.bodies[0].kinematic = 1
    g = run_gpu(lbib, case, 25)
    o = run_oracle(case, 25)
    check_fp64(g, o)


def test_fp64_momentum_exchange_rigid_bodies(lbib):
    """Momentum-exchange rigid-body force variant: a heavy sphere settling in
    a walled box and a free sphere in Couette flow, 30 steps."""
    v, f = W.icosphere(3, 3.5, (10.0, 11.0, 17.0))
    settle = W.Case("settle_mx", (20, 22, 30), 0.7, (W.WALL, W.WALL, W.WALL), np.zeros((6, 3)),
                    precision=W.PREC_FP64, bodies=[W.Body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.5,
                                                          gravity=(0.0, 0.0, -2e-5), rigid_force=1)])
    couette = W.case_couette_sphere()
    couette.bodies[0].rigid_force = 1
    for case in (settle, couette):
        g = run_gpu(lbib, case, 30)
        o = run_oracle(case, 30)
        check_fp64(g, o)


def centroid_cases():
    """Centroid IB markers on every body kind: a perturbed capsule in shear
    (dynamic and kinematic), a heavy sphere settling in a walled box (both
    rigid-body force readings) and the free sphere in Couette flow."""
    out = []
    for kinematic in (0, 1):
        case = W.case_capsule_shear(n=24, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                    kv=1.0, precision=W.PREC_FP64)
        case.bodies[0].verts = W.perturb(case.bodies[0].verts, 0.02, seed=11)
        case.bodies[0].kinematic = kinematic
        out.append(case)
    v, f = W.icosphere(3, 3.5, (10.0, 11.0, 17.0))
    for rigid_force in (0, 1):
        out.append(W.Case("settle_c", (20, 22, 30), 0.7, (W.WALL, W.WALL, W.WALL), np.zeros((6, 3)),
                          precision=W.PREC_FP64,
                          bodies=[W.Body(v, f, rigid=True, density_ratio=1.5, ref_radius=3.5,
                                         gravity=(0.0, 0.0, -2e-5), rigid_force=rigid_force)]))
    out.append(W.case_couette_sphere())
    for case in out:
        case.bodies[0].centroid_markers = 1
    return out


@pytest.mark.parametrize("k", range(5))
def test_fp64_centroid_markers(lbib, k):
    case = centroid_cases()[k]
    g = run_gpu(lbib, case, 30)
    o = run_oracle(case, 30)
    check_fp64(g, o)
    if case.bodies[0].rigid:
        # omega of the settling sphere is round-off of cancelling moments:
        # held on the scale u / R of the body's motion
        bg, bo = g["bodies"][0], o["bodies"][0]
        scale = max(np.abs(bo["u"]).max(), np.abs(bo["omega"]).max() * case.bodies[0].ref_radius)
        assert np.abs(bg["u"] - bo["u"]).max() <= 1e-12 * scale
        assert np.abs(bg["omega"] - bo["omega"]).max() * case.bodies[0].ref_radius <= 1e-12 * scale


def test_fp64_two_bodies_and_gravity_periodic(lbib):
    """Two bodies in one periodic lattice: a settling rigid sphere and a
    capsule (shared force field, several spreads per step)."""
    n = (26, 22, 30)
    v1, f1 = W.icosphere(2, 3.0, (7.2, 10.9, 20.1))
    v2, f2 = W.icosphere(2, 3.5, (18.4, 11.3, 9.7))
    case = W.Case("two_bodies", n, 0.7, (0, 0, 0), np.zeros((6, 3)), precision=W.PREC_FP64, steps=30,
                  bodies=[W.Body(v1, f1, rigid=True, density_ratio=1.3, ref_radius=3.0, gravity=(0, 0, -2e-5)),
                          W.Body(v2, f2, ks0=5e-3, Eb=0.02, kv=1.0, density_ratio=2.0, ref_radius=3.5)])
    g = run_gpu(lbib, case, 30)
    o = run_oracle(case, 30)
    check_fp64(g, o)


# ---------------------------------------------------------------------------------------
# FP32 at the benchmark sizes
# ---------------------------------------------------------------------------------------

def check_fp32(g, o, pos_tol=1e-4, vel_tol=1e-5):
    ug, uo = g["fields"][1], o["fields"][1]
    assert rel(ug, uo) < vel_tol
    assert np.abs(g["fields"][0] - o["fields"][0]).max() < 1e-6
    for (Xg, _, _), (Xo, _, _) in zip(g["markers"], o["markers"]):
        assert np.abs(Xg - Xo).max() < pos_tol


@pytest.mark.parametrize("Ca,Eb", [(0.01, 0.005), (0.05, 0.01), (0.2, 0.01)])
def test_fp32_capsule_96_full_size(lbib, Ca, Eb):
    """96^3 capsule in shear (radius 10, 2562 markers, 5120 triangles),
    tau 0.8, shear rate 1e-4, FP32 storage and arithmetic, 60 steps.  At
    Ca = 0.01 the bending ratio is 0.005: with 0.01 the stiffest bending mode
    leaves the stability region of the explicit marker update (the oracle
    diverges as well)."""
    case = W.case_capsule_shear(Ca=Ca, Eb=Eb, kv=1.0)
    g = run_gpu(lbib, case, 60)
    o = run_oracle(case, 60)
    check_fp32(g, o)


def test_fp32_capsule_96_centroid_markers(lbib):
    """The 96^3 capsule (Ca 0.05) with its IB markers at the 5120 triangle
    centroids, FP32, 60 steps."""
    case = W.case_capsule_shear(Ca=0.05, Eb=0.01, kv=1.0)
    case.bodies[0].centroid_markers = 1
    g = run_gpu(lbib, case, 60)
    o = run_oracle(case, 60)
    check_fp32(g, o)


def test_fp32_settling_box_full_size(lbib):
    """160x160x480 walled box, rigid sphere radius 8 (10242 markers), tau 0.7,
    FP32, 3 steps; fields and markers."""
    case = W.case_settling()
    g = run_gpu(lbib, case, 3)
    o = run_oracle(case, 3)
    check_fp32(g, o)


def test_overlapped_and_serial_sweeps_agree(lbib):
    """The far-field sweep on the second stream plus the box sweep equals one
    whole-lattice sweep (FP64; only the order of the atomic spreading sums
    may differ)."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    out = []
    for overlap in (1, 0):
        ctx = lbib.Context.from_case(case)
        lbib.lbib_set_overlap(ctx.h, overlap)
        ctx.step(25)
        out.append((ctx.populations(), ctx.markers(0)[0]))
        ctx.close()
    assert rel(out[0][0], out[1][0]) < 1e-14
    assert rel(out[0][1], out[1][1]) < 1e-14


@pytest.mark.parametrize("overlap", [1, 0])
def test_graph_steps_match_enqueued_steps(lbib, overlap):
    """Steps replayed from the six captured CUDA graphs equal steps whose
    kernels are enqueued one by one (FP64; only the order of the atomic
    spreading sums may differ, hence 1e-13), also when field-storing steps, which are
    enqueued directly, interleave with graph steps at every phase of the
    buffer rotation."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    out = []
    for graphs in (1, 0):
        ctx = lbib.Context.from_case(case)
        lbib.lbib_set_overlap(ctx.h, overlap)
        lbib.lbib_set_graphs(ctx.h, graphs)
        lbib.lbib_set_output(ctx.h, 5)
        for n in (7, 1, 6, 11):
            ctx.step(n)
        out.append((ctx.populations(), ctx.markers(0)[0], ctx.fields()[1]))
        ctx.close()
    for a, b in zip(out[0], out[1]):
        assert rel(a, b) < 1e-13
    o = run_oracle(case, 25)
    assert rel(out[0][0], o["f"]) < 1e-12


@pytest.mark.parametrize("config", [(1, 0, 0, 0), (0, 32, 4, 0), (0, 128, 2, 0), (0, 0, 0, 1), (0, 32, 4, 2)])
@pytest.mark.parametrize("overlap", [1, 0])
def test_sweep_kernels_and_shapes_match_oracle(lbib, config, overlap):
    """The row-tile sweep (x-rows staged in shared memory, 128-bit loads
    and stores) and the one-node sweep in several block shapes compute the
    same steps (FP64, 28^3 capsule in shear, with and without the far-field
    sweep running beside the IB stage)."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    ctx = lbib.Context.from_case(case)
    lbib.lbib_set_sweep_config(ctx.h, *config)
    lbib.lbib_set_overlap(ctx.h, overlap)
    ctx.step(20)
    g = {"f": ctx.populations(), "fields": ctx.fields(), "markers": [ctx.markers(0)]}
    ctx.close()
    check_fp64(g, run_oracle(case, 20))


def test_fp32_row_tile_sweep_full_size(lbib):
    """The row-tile kernel on the 96^3 FP32 capsule case against the oracle."""
    case = W.case_capsule_shear(Ca=0.05, Eb=0.01, kv=1.0)
    ctx = lbib.Context.from_case(case)
    lbib.lbib_set_sweep_config(ctx.h, 1, 0, 0, 2)
    ctx.step(30)
    g = {"fields": ctx.fields(), "markers": [ctx.markers(0)]}
    ctx.close()
    check_fp32(g, run_oracle(case, 30))


def test_autotuned_launch_configurations_keep_parity(lbib):
    """Every block shape and overlap mode the autotuner tries computes the
    same step: after tuning (which advances the run) the state still matches
    the oracle advanced by the same number of steps."""
    case = W.case_capsule_shear(n=26, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    ctx = lbib.Context.from_case(case)
    choice = lbib.lbib_autotune(ctx.h, 1)
    assert choice[2] in (0, 1) and lbib.lbib_get_launch_config(ctx.h)[5] in (0, 1, 2)
    ctx.step(4)
    nsteps, _ = ctx.counters()
    g = {"f": ctx.populations(), "fields": ctx.fields(), "markers": [ctx.markers(0)]}
    ctx.close()
    o = run_oracle(case, nsteps)
    check_fp64(g, o)


@pytest.mark.parametrize("rigid", [False, True])
def test_ib_block_cap_keeps_parity(lbib, rigid):
    """lbib_set_ib_blocks: the MLS, structure and spreading kernels on one
    block per SM, each block taking several groups of points, markers or
    vertices in turn (2562 markers and 10240 probes: 401 MLS and 321 marker
    groups), compute the steps of their full grids (FP64, up to the order of
    the spreading sums), and the rigid sphere's match the oracle.  (This
    sphere is centred on a half-integer, so 606 of its markers and probes
    start exactly on a cell boundary, floor(X + 1/2) at an integer; after a
    step, 1e-16 of position decides their support node, and the membrane's
    GPU and oracle runs part at the 1e-12 level for that reason alone.)"""
    case = W.case_capsule_shear(n=40, tau=0.8, shear_rate=2e-3, radius=8.0, level=4, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    if rigid:
        b = case.bodies[0]
        case.bodies = [W.Body(b.verts, b.tris, rigid=True, density_ratio=1.0, ref_radius=8.0)]
    runs = []
    for cap in (0, 1):
        ctx = lbib.Context.from_case(case)
        lbib.lbib_set_ib_blocks(ctx.h, cap)
        assert lbib.lbib_get_launch_config(ctx.h)[5] == cap
        ctx.step(10)
        runs.append({"f": ctx.populations(), "fields": ctx.fields(), "markers": [ctx.markers(0)]})
        if cap:
            with pytest.raises(lbib.LbibError):
                lbib.lbib_set_ib_blocks(ctx.h, -1)
        ctx.close()
    check_fp64(runs[1], runs[0], tol=1e-14)
    if rigid:
        check_fp64(runs[1], run_oracle(case, 10))


@pytest.mark.parametrize("prec,tol", [(W.PREC_FP64, 1e-15), (W.PREC_FP32, 1e-7)])
def test_shear_fields_are_the_couette_equilibrium(lbib, prec, tol):
    """lbib_set_shear_fields forms on the device the equilibrium of the
    linear shear profile between the z walls, the same populations as
    setting that profile as host fields; the state is then the exact
    discrete steady state (100 steps leave it within rounding)."""
    n, U = (6, 5, 24), 0.01
    a = lbib.Context(n, 0.8, bc=(0, 0, 1), wall_u=W.shear_walls(U), precision=prec)
    lbib.lbib_set_shear_fields(a.h, -U, U)
    b = lbib.Context(n, 0.8, bc=(0, 0, 1), wall_u=W.shear_walls(U), precision=prec)
    b.set_fields(np.ones(n[0] * n[1] * n[2]), W.couette_profile(n, U))
    fa, fb = a.populations(), b.populations()
    assert rel(fa, fb) < tol
    a.step(100)
    _, u = a.fields()
    assert np.abs(u - W.couette_profile(n, U)).max() < 100 * tol * U
    with pytest.raises(lbib.LbibError):
        lbib.lbib_set_shear_fields(a.h, float("nan"), U)
    a.close()
    b.close()


@pytest.mark.parametrize("tau", [0.8, 0.7, 0.6])
def test_fp32_collision_returns_the_momentum_it_is_given(lbib, tau):
    """A periodic box without force keeps its total momentum exactly; in
    FP32 the collision's odd part, formed from the momentum with
    coefficients whose momentum sums to omega exactly, leaves the rounding
    of the moment sums and the stores: drift over these 2000 steps 1.9e-6,
    1.2e-6, 2.8e-6 of the momentum's size at tau 0.8, 0.7, 0.6.  Formed
    from the rounded velocity with the rounded weights 1/18 and 1/36 the
    collision returned the momentum times (1 + ~1e-8) at every step: drift
    1.5e-5, 1.5e-4, 1.0e-4.  The bound is 6e-6."""
    case = W.case_empty(n=(24, 20, 16), tau=tau, precision=W.PREC_FP32, seed=21, amplitude=1e-2)
    case.u0 = case.u0 + np.array([3e-3, -2e-3, 1e-3])  # a mean flow on top of the random field
    ctx = lbib.Context.from_case(case)
    _, p0 = lbib.lbib_get_totals(ctx.h)
    ctx.step(2000)
    _, p1 = lbib.lbib_get_totals(ctx.h)
    ctx.close()
    assert np.abs(p1 - p0).max() < 6e-6 * np.abs(p0).max(), (p0, p1)


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [(W.PREC_FP64, 1e-12), (W.PREC_FP32, 2e-6)])
def test_fp64_totals_conservation_and_forcing(lbib, prec, tol, paper_e):
    """The GPU's FP64 mass/momentum reduction: on a periodic lattice the
    mass is constant and the momentum grows by exactly ncell * g_ext per step
    (streaming conserves both; the Guo collision adds the force, Eq.
    forcing), and at the end both equal the sums over the oracle's
    populations.  FP32 storage: within its rounding."""
    g = np.array([2e-6, -1e-6, 5e-7])
    case = W.case_empty(n=(33, 17, 12), tau=0.7, gext=tuple(g), precision=prec, seed=11)
    ctx = lbib.Context.from_case(case)
    m0, p0 = lbib.lbib_get_totals(ctx.h)
    nc = case.ncell
    for k in range(1, 4):
        ctx.step(5)
        m, p = lbib.lbib_get_totals(ctx.h)
        assert abs(m - m0) <= tol * nc
        assert np.abs(p - p0 - 5 * k * nc * g).max() <= tol * nc * 1e-2
    f = ctx.populations()
    ctx.close()
    o = run_oracle(case, 15)["f"]
    assert abs(m - o.sum()) <= tol * nc
    assert np.abs(p - (o @ paper_e).sum(axis=0)).max() <= tol * nc * 1e-2


def test_checkpoint_resume_continues_the_run(lbib):
    """Save after 9 steps, run 7 more; a freshly set-up context loaded from
    the checkpoint runs the same 7 steps to the same state (FP64; only the
    order of the atomic spreading sums may differ).  A checkpoint of a
    different set-up is refused; loading clears a sticky error."""
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    a = lbib.Context.from_case(case)
    a.step(9)
    ck = lbib.lbib_save(a.h)
    a.step(7)
    fa, Xa = a.populations(), a.markers(0)[0]
    b = lbib.Context.from_case(case)
    lbib.lbib_load(b.h, ck)
    assert b.counters()[0] == 9
    b.step(7)
    assert rel(b.populations(), fa) < 1e-13 and rel(b.markers(0)[0], Xa) < 1e-13
    other = lbib.Context((28, 28, 30), 0.8, bc=(0, 0, 1), precision=lbib.LBIB_FP64)
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_load(other.h, ck)
    assert ei.value.code == lbib.LBIB_EINVAL
    other.close()
    # a sticky error (support reaching a wall) is cleared by loading the
    # checkpoint of a context set up the same way with the sphere clear of
    # the walls
    n = 16
    ctxs = []
    for zc in (8.0, 3.2):
        v, f = W.icosphere(1, 2.0, (8.0, 8.0, zc))
        ctx = lbib.Context((n, n, n), 0.8, bc=(0, 0, 1), precision=lbib.LBIB_FP64)
        ctx.add_body(v, f, rigid=True, ref_radius=2.0)
        ctxs.append(ctx)
    good = lbib.lbib_save(ctxs[0].h)
    c = ctxs[1]
    with pytest.raises(lbib.LbibError) as ei:
        c.step(1)
        c.sync()
    assert ei.value.code == lbib.LBIB_EBODY_WALL
    lbib.lbib_load(c.h, good)
    c.step(2)
    c.sync()
    assert abs(c.markers(0)[0][:, 2].mean() - 8.0) < 1e-6
    ctxs[0].close()
    for ctx in (a, b, c):
        ctx.close()


def test_async_marker_copies_are_ordered_on_the_stream(lbib):
    """lbib_get_markers_async queued after step 3 returns the markers of
    step 3 although two more steps are queued before the synchronisation
    (page-locked and pageable host arrays): the values a synchronous read
    gave at step 3."""
    case = W.case_capsule_shear(n=24, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    nv = case.bodies[0].verts.shape[0]
    ctx = lbib.Context.from_case(case)
    ctx.step(3)
    X3, V3, F3 = ctx.markers(0)
    pinned = [torch.empty((nv, 3), dtype=torch.float64, pin_memory=True) for _ in range(3)]
    lbib.lbib_get_markers_async(ctx.h, 0, *pinned)
    pageable = [np.full((nv, 3), np.nan) for _ in range(3)]
    lbib.lbib_get_markers_async(ctx.h, 0, *pageable)
    ctx.step(2)
    lbib.lbib_sync(ctx.h)
    for got in (pinned, pageable):
        for a, b in zip(got, (X3, V3, F3)):
            assert np.array_equal(np.asarray(a), b)
    assert not np.array_equal(ctx.markers(0)[0], X3)  # the context went on to step 5
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_get_markers_async(ctx.h, 1, *pageable)
    assert ei.value.code == lbib.LBIB_EINVAL
    ctx.close()


def test_recorded_trajectory_matches_step_by_step_reads(lbib):
    """lbib_step_markers: calls of 5, 9 (the device staging buffer grows), 2
    and 0 steps with every step's markers recorded into host rings (pinned
    and pageable; V omitted in one call), against a context read
    synchronously after each step (the two differ only in the order of the
    atomic spreading sums)."""
    case = W.case_capsule_shear(n=24, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=W.PREC_FP64)
    nv = case.bodies[0].verts.shape[0]
    calls = [5, 9, 2, 0]
    ref = lbib.Context.from_case(case)
    want = []
    for k in range(sum(calls)):
        ref.step(1)
        want.append(ref.markers(0))
    ref.close()
    ctx = lbib.Context.from_case(case)
    done = 0
    for j, n in enumerate(calls):
        X = torch.empty((max(n, 1), nv, 3), dtype=torch.float64, pin_memory=True)
        V = np.full((max(n, 1), nv, 3), np.nan)
        F = np.full((max(n, 1), nv, 3), np.nan)
        lbib.lbib_step_markers(ctx.h, n, 0, X, V if j != 0 else None, F)
        lbib.lbib_sync(ctx.h)
        for k in range(n):
            Xw, Vw, Fw = want[done + k]
            assert rel(X[k].numpy(), Xw) < 1e-13
            if j != 0:
                assert np.abs(V[k] - Vw).max() < 1e-10 * max(np.abs(Vw).max(), 1e-3)
            assert np.abs(F[k] - Fw).max() < 1e-10 * max(np.abs(Fw).max(), 1e-3)
        if j == 0:
            assert np.isnan(V).all()
        done += n
    assert ctx.counters()[0] == sum(calls)
    ctx.close()


def test_zero_steps_and_empty_lattice(lbib):
    case = W.case_empty(n=(5, 4, 3), precision=W.PREC_FP64, seed=7)
    ctx = lbib.Context.from_case(case)
    ctx.step(0)
    rho, u = ctx.fields()
    r0, u0 = case.initial_fields()
    assert np.abs(rho - r0).max() < 1e-15 and np.abs(u - u0).max() < 1e-15
    ctx.close()


def test_support_reaching_wall_reports_error(lbib):
    n = 16
    v, f = W.icosphere(1, 2.0, (8.0, 8.0, 3.2))
    ctx = lbib.Context((n, n, n), 0.8, bc=(0, 0, 1), precision=lbib.LBIB_FP64)
    ctx.add_body(v, f, rigid=True, ref_radius=2.0)
    ctx.step(1)
    with pytest.raises(lbib.LbibError) as ei:
        ctx.sync()
    assert ei.value.code == lbib.LBIB_EBODY_WALL
    with pytest.raises(lbib.LbibError):
        ctx.step(1)  # sticky
    ctx.close()


def test_invalid_bodies_rejected(lbib):
    ctx = lbib.Context((16, 16, 16), 0.8, precision=lbib.LBIB_FP32)
    v, f = W.icosphere(1, 3.0, (8, 8, 8))
    with pytest.raises(lbib.LbibError):
        ctx.add_body(v, f[:-1])  # open mesh
    with pytest.raises(lbib.LbibError):
        ctx.add_body(v, f[:, ::-1].copy())  # inward orientation
    with pytest.raises(lbib.LbibError):
        ctx.add_body(v, f, density_ratio=0.0)
    ctx.close()


@pytest.mark.parametrize("nz", [592, 600])
def test_plane_offsets_at_the_32_bit_limit(lbib, nz):
    """The sweep forms population addresses with 32-bit plane offsets while
    all 19 planes lie within 2^32 elements of the first, and in 64 bits
    above that.  616 x 616 x 592 (224.6 M nodes) is just below the limit,
    616 x 616 x 600 (227.7 M nodes) just above it.  A periodic FP32 lattice
    filled with copies of a random 8^3 state evolves exactly as the 8^3
    lattice does (every copy sees the same neighbours and the arithmetic per
    node is the same), so after three steps the fields of every node equal
    those of the small lattice bit for bit: an offset that wraps or a plane
    addressed from the wrong base would differ at the size of the flow."""
    small = W.case_empty(n=(8, 8, 8), tau=0.8, precision=W.PREC_FP32, seed=11, amplitude=2e-2)
    ctx = lbib.Context.from_case(small)
    ctx.step(3)
    rho_s, u_s = ctx.fields()
    ctx.close()
    n = (616, 616, nz)
    assert (19 * ((n[0] * n[1] * n[2] + 63) // 64 * 64) > 2 ** 32) == (nz == 600)
    reps = (nz // 8, n[1] // 8, n[0] // 8)
    rho0, u0 = small.initial_fields()
    dev = torch.device("cuda")
    rho = torch.from_numpy(rho0.reshape(8, 8, 8)).to(dev).repeat(*reps).contiguous()
    u = torch.from_numpy(u0.reshape(8, 8, 8, 3)).to(dev).repeat(*reps, 1).contiguous()
    h = lbib.lbib_create(lbib.make_params(n, 0.8, bc=(W.PERIODIC,) * 3, precision=lbib.LBIB_FP32))
    try:
        torch.cuda.synchronize()
        lbib.lbib_set_fields(h, rho, u)
        del rho, u
        lbib.lbib_step(h, 3)
        rho_b = torch.empty(n[0] * n[1] * n[2], dtype=torch.float64, device=dev)
        u_b = torch.empty(3 * n[0] * n[1] * n[2], dtype=torch.float64, device=dev)
        lbib.lbib_get_fields(h, rho_b, u_b)
        torch.cuda.synchronize()
    finally:
        lbib.lbib_destroy(h)
    want_rho = torch.from_numpy(rho_s.reshape(8, 8, 8)).to(dev).repeat(*reps).reshape(-1)
    assert torch.equal(rho_b, want_rho)
    del rho_b, want_rho
    want_u = torch.from_numpy(u_s.reshape(8, 8, 8, 3)).to(dev).repeat(*reps, 1).reshape(-1)
    assert torch.equal(u_b, want_u)
    del u_b, want_u
    torch.cuda.empty_cache()


def test_add_body_rejects_meshes_that_are_not_closed_oriented_manifolds(lbib):
    """The hinge set-up needs every directed edge once and its twin: an
    open mesh, a repeated triangle (its directed edges twice) and an inward
    orientation (negative enclosed volume) are LBIB_EINVAL, and the context
    stays usable."""
    v, f = W.icosphere(2, 4.0, (8.0, 8.0, 8.0))
    ctx = lbib.Context((16, 16, 16), 0.8, precision=lbib.LBIB_FP64)
    for bad in (f[1:], np.concatenate([f, f[:1]]), f[:, ::-1].copy()):
        with pytest.raises(lbib.LbibError) as ei:
            ctx.add_body(v, bad, **W.Body(v, bad, ks0=1e-3, ref_radius=4.0).kwargs())
        assert ei.value.code == lbib.LBIB_EINVAL
    ctx.add_body(v, f, **W.Body(v, f, ks0=1e-3, ref_radius=4.0).kwargs())
    ctx.step(2)
    assert np.isfinite(ctx.markers(0)[0]).all()
    ctx.close()
