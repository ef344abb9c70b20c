"""Writes fp32_long_refs/*.npz: the FP64 oracle's state after the stated step
counts of the two FP32 benchmark cases, against which the long FP32 parity
tests compare the GPU path.  Calls only the oracle (and the seeded case
builders, which hold no method arithmetic).

- 96^3 capsule in shear (radius 10, 2562 markers), Ca 0.01 / 0.05 / 0.2:
  checkpoints at 2000 and 20000 steps (the stated run length).
- 160x160x480 settling sphere (radius 8, 10242 markers): checkpoints at 100
  and 300 steps.

Each checkpoint stores every marker position and the density and velocity of
the last collision at a fixed sample of nodes: SAMPLE_UNIFORM nodes drawn
uniformly over the lattice and SAMPLE_NEAR nodes drawn from the box of half
width 1.5 radii around the body's starting centre (seeded; the node indices
are stored beside the values).

    OMP_NUM_THREADS=8 python tests/golden/make_fp32_long_refs.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2207_06029_gb300 import workloads as W  # noqa: E402

OUT_DIR = os.path.join(HERE, "fp32_long_refs")
SAMPLE_UNIFORM = 4096
SAMPLE_NEAR = 4096

# name -> (case builder, checkpoints); the builders are the ones the tests use
CASES = {
    "capsule96_Ca0.01": (lambda: W.case_capsule_shear(Ca=0.01, Eb=0.005, kv=1.0, precision=W.PREC_FP64),
                         (2000, 20000)),
    "capsule96_Ca0.05": (lambda: W.case_capsule_shear(Ca=0.05, Eb=0.01, kv=1.0, precision=W.PREC_FP64),
                         (2000, 20000)),
    "capsule96_Ca0.2": (lambda: W.case_capsule_shear(Ca=0.2, Eb=0.01, kv=1.0, precision=W.PREC_FP64),
                        (2000, 20000)),
    "settling160x160x480": (lambda: W.case_settling(precision=W.PREC_FP64), (100, 300)),
}


def sample_nodes(case, seed=2207):
    """Node indices (x fastest) of the sample: uniform over the lattice plus
    uniform over the box around the body's starting centre."""
    nx, ny, nz = case.n
    rng = np.random.default_rng(seed)
    uni = rng.integers(0, case.ncell, SAMPLE_UNIFORM)
    v = case.bodies[0].verts
    c = v.mean(axis=0)
    r = 1.5 * np.abs(v - c).max()
    lo = np.maximum(np.floor(c - r), 0).astype(int)
    hi = np.minimum(np.ceil(c + r), np.array(case.n) - 1).astype(int)
    pts = np.stack([rng.integers(lo[a], hi[a] + 1, SAMPLE_NEAR) for a in range(3)], axis=1)
    near = pts[:, 0] + nx * (pts[:, 1] + ny * pts[:, 2])
    return np.unique(np.concatenate([uni, near])).astype(np.int64)


def run(name):
    build, checkpoints = CASES[name]
    case = build()
    idx = sample_nodes(case)
    s = oracle.Sim(case.n, case.tau, gext=case.gext, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    for b in case.bodies:
        s.add_body(b.verts, b.tris, **b.kwargs())
    out = {"nodes": idx}
    done = 0
    t0 = time.time()
    for k in checkpoints:
        rc = s.step(k - done)
        assert rc == 0, f"{name}: oracle returned {rc} before step {k}"
        done = k
        rho, u = s.fields()
        X, _, _ = s.markers(0)
        out[f"rho_{k}"] = rho[idx]
        out[f"u_{k}"] = u.reshape(-1, 3)[idx]
        out[f"X_{k}"] = X
        print(f"{name}: step {k} after {time.time() - t0:.0f} s", flush=True)
    s.close()
    out["checkpoints"] = np.array(checkpoints, np.int64)
    os.makedirs(OUT_DIR, exist_ok=True)
    np.savez_compressed(os.path.join(OUT_DIR, f"{name}.npz"), **out)


def main(names):
    for name in names or list(CASES):
        run(name)


if __name__ == "__main__":
    main(sys.argv[1:])
