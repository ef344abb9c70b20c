"""Writes reduced_precision_refs.txt: the FP64 oracle's Taylor deformation
D(t) of the capsule-in-shear case (every 50 steps up to 2000) and the
quarter period of the Jeffery-orbit case, against which the reduced-precision
storage tests compare.  Calls only the oracle.

    python tests/golden/make_reduced_precision_refs.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2207_06029_gb300 import workloads as W  # noqa: E402
from test_gpu_reduced_precision import (CAPSULE, D_EVERY, D_STEPS, JEFFERY_EVERY, JEFFERY_STEPS,  # noqa: E402
                                        major_axis_x, quarter_period, taylor_D)


def sim(case):
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    for b in case.bodies:
        s.add_body(b.verts, b.tris, **b.kwargs())
    return s


def main():
    lines = ["# FP64 oracle references of the reduced-precision storage tests",
             "# written by make_reduced_precision_refs.py (oracle only)"]
    case = W.case_capsule_shear(precision=W.PREC_FP64, **CAPSULE)
    s = sim(case)
    for k in range(D_EVERY, D_STEPS + 1, D_EVERY):
        assert s.step(D_EVERY) == 0
        lines.append(f"D {k} {taylor_D(s.markers(0)[0], case.bodies[0].tris):.12e}")
    s.close()
    case = W.case_jeffery_spheroid(precision=W.PREC_FP64)
    s = sim(case)
    samples = [(0, 1.0)]
    for k in range(JEFFERY_EVERY, JEFFERY_STEPS + 1, JEFFERY_EVERY):
        assert s.step(JEFFERY_EVERY) == 0
        samples.append((k, major_axis_x(s.body(0)["q"])))
    s.close()
    lines.append(f"T4 {quarter_period(samples):.12e}")
    with open(os.path.join(HERE, "reduced_precision_refs.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
