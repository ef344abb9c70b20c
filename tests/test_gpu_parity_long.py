"""FP32 GPU path against the FP64 oracle after the stated run lengths.

The oracle's state at fixed checkpoints of the two FP32 benchmark cases is
stored in tests/golden/fp32_long_refs/ by tests/golden/make_fp32_long_refs.py
(oracle only): every marker position and the density and velocity of the
last collision at a seeded sample of nodes (uniform over the lattice plus
the neighbourhood of the body).  The GPU runs the same case in FP32 storage
and arithmetic and is compared at every checkpoint:

- velocity: max |u_gpu - u_oracle| / max |u_oracle| over the sample < 1e-5;
- density: max |rho_gpu - rho_oracle| < 1e-6;
- marker positions: max |X_gpu - X_oracle| < 1e-4 lattice units.

96^3 capsule in shear (Ca 0.01, 0.05, 0.2): 2000 and 20000 steps (the
stated run length, a dimensionless time shear_rate * t = 2).
160x160x480 settling sphere: 100 and 300 steps.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_fp32_long_refs as refs  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VEL_TOL, RHO_TOL, POS_TOL = 1e-5, 1e-6, 1e-4


@pytest.fixture(scope="module")
def lbib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06029_gb300 import build, lbib as L
    build.build()
    L.load()
    return L


@pytest.mark.parametrize("name", sorted(refs.CASES))
def test_fp32_after_the_stated_steps(lbib, name):
    path = os.path.join(refs.OUT_DIR, f"{name}.npz")
    ref = np.load(path)
    build, checkpoints = refs.CASES[name]
    case = build()
    nodes = ref["nodes"]
    assert np.array_equal(nodes, refs.sample_nodes(case))
    ctx = lbib.Context.from_case(case, precision=lbib.LBIB_FP32)
    done = 0
    report = []
    for k in checkpoints:
        ctx.step(k - done)
        done = k
        rho, u = ctx.fields()
        X = ctx.markers(0)[0]
        u_ref, rho_ref, X_ref = ref[f"u_{k}"], ref[f"rho_{k}"], ref[f"X_{k}"]
        err_u = np.abs(u[nodes] - u_ref).max() / np.abs(u_ref).max()
        err_rho = np.abs(rho[nodes] - rho_ref).max()
        err_X = np.abs(X - X_ref).max()
        report.append((k, err_u, err_rho, err_X))
    ctx.close()
    print(name, " ".join(f"step {k}: u {eu:.2e} rho {er:.2e} X {ex:.2e}" for k, eu, er, ex in report))
    for k, err_u, err_rho, err_X in report:
        assert err_u < VEL_TOL, (k, err_u)
        assert err_rho < RHO_TOL, (k, err_rho)
        assert err_X < POS_TOL, (k, err_X)
