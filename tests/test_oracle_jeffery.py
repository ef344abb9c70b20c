"""Jeffery orbit of a rigid prolate spheroid in shear (the oracle's rigid
body, probes and coupling together).

Jeffery (1922): a neutrally buoyant spheroid of aspect ratio r with its axis
in the shear plane turns with period T = 2 pi (r + 1/r) / shear_rate in
unbounded Stokes flow; the axis passes the wall normal after T/4.  Finite
Reynolds number and the walls both slow the rotation, so on a lattice the
quarter period lies above Jeffery's and approaches it as the box grows and
the shear rate falls.  Aspect ratio 2 (semi-axes 6, 3, 3): Re = 7.2 in the
32^3 box, 3.6 in the 48^3 box.
"""
import math

import oracle
from paper_2207_06029_gb300 import workloads as W


def quarter_period(n, shear_rate):
    case = W.case_jeffery_spheroid(n=n, shear_rate=shear_rate, precision=W.PREC_FP64)
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    prev_t, prev_d, k = 0, 1.0, 0
    limit = 2.0 * math.pi * 2.5 / (2.0 * shear_rate)
    while k < limit:
        assert s.step(20) == 0
        k += 20
        w, x, y, z = s.body(0)["q"]
        d = 1.0 - 2.0 * (y * y + z * z)  # x-component of the body's major axis
        if d <= 0.0:
            s.close()
            return prev_t + (k - prev_t) * prev_d / (prev_d - d)
        prev_t, prev_d = k, d
    s.close()
    raise AssertionError("no quarter turn")


def test_quarter_period_approaches_jeffery():
    excess = []
    for n, g in ((32, 5e-3), (48, 2.5e-3)):
        jeffery = math.pi * (2.0 + 0.5) / (2.0 * g)
        excess.append(quarter_period(n, g) / jeffery - 1.0)
    assert excess[0] > excess[1] > 0.0  # slower than Stokes flow, less so in the larger box
    assert excess[1] < 0.15
