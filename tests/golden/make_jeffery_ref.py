"""Writes jeffery_oracle_ref.txt: the FP64 oracle's Jeffery quarter period of
a resolved rigid prolate spheroid in shear, the case the paper validates its
rigid-body coupling with (Sec. 3.3).  Calls only the oracle (and the seeded
case builder, which holds no method arithmetic).

Spheroid of aspect ratio 2, semi-axes (12, 6, 6) (icosphere level 4, 2562
markers), neutrally buoyant, at the centre of a 120^3 Couette cell with z
walls (confinement 2a/H = 0.2), tau 0.8, shear rate 0.2 nu / a^2 (particle
Reynolds number shear a^2 / nu = 0.2), the printed stress-jump force.  The
quarter period is the step at which the major axis passes the wall normal
(linear interpolation between samples every 50 steps), divided by Jeffery's
T/4 = pi (r + 1/r) / (2 shear).

    OMP_NUM_THREADS=8 python tests/golden/make_jeffery_ref.py
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2207_06029_gb300 import workloads as W  # noqa: E402

A, N, TAU, RE, LEVEL, EVERY = 12.0, 120, 0.8, 0.2, 4, 50


def case():
    nu = (TAU - 0.5) / 3.0
    shear = RE * nu / A ** 2
    return W.case_jeffery_spheroid(n=N, tau=TAU, shear_rate=shear, axes=(A, A / 2, A / 2), level=LEVEL,
                                   precision=W.PREC_FP64), shear


def main():
    c, shear = case()
    s = oracle.Sim(c.n, c.tau, gext=c.gext, bc=c.bc, wall_u=c.wall_u.ravel())
    s.set_fields(*c.initial_fields())
    b = c.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    jeffery = math.pi * 2.5 / (2.0 * shear)
    prev_t, prev_d, k, t0 = 0, 1.0, 0, time.time()
    while True:
        assert s.step(EVERY) == 0
        k += EVERY
        w, x, y, z = s.body(0)["q"]
        d = 1.0 - 2.0 * (y * y + z * z)  # x-component of the major axis
        if k % 5000 == 0:
            print(f"step {k}: axis x {d:.6f} after {time.time() - t0:.0f} s", flush=True)
        if d <= 0.0:
            t4 = prev_t + (k - prev_t) * prev_d / (prev_d - d)
            break
        prev_t, prev_d = k, d
        assert k < 2 * jeffery, "no quarter turn"
    s.close()
    with open(os.path.join(HERE, "jeffery_oracle_ref.txt"), "w") as fh:
        fh.write("# FP64 oracle: Jeffery quarter period of a rigid prolate spheroid (12, 6, 6) in a 120^3\n"
                 "# Couette cell, tau 0.8, Re 0.2, stress-jump force; written by make_jeffery_ref.py (oracle only)\n")
        fh.write(f"quarter_period_steps {t4:.6f}\n")
        fh.write(f"jeffery_quarter_period_steps {jeffery:.6f}\n")
        fh.write(f"ratio {t4 / jeffery:.8f}\n")


if __name__ == "__main__":
    main()
