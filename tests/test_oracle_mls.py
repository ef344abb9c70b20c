"""Pins of the oracle's moving-least-squares transfer (Sec. 2.2).

References: the consistency conditions a linear-basis least-squares fit must
satisfy (partition of unity, reproduction of linear fields and of their
gradients), a closed form for a marker sitting on a node, the printed
support constants, and conservation/adjointness of interpolation and
spreading inside a full step.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2207_06029_gb300 import workloads as W


def _nodes(base):
    k = np.arange(27)
    d = np.stack([k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1], axis=1)
    return base[None, :] + d


@pytest.mark.parametrize("seed", range(4))
def test_mls_consistency(seed):
    """Linear basis: sum phi = 1, sum phi x_k = X, and the full fit reproduces
    any linear field a + G x exactly, value and gradient."""
    rng = np.random.default_rng(seed)
    for _ in range(250):
        X = rng.uniform(-20, 20, 3)
        base, psi = oracle.mls_point(X)
        xk = _nodes(base).astype(np.float64)
        phi = psi[:, 0]
        assert abs(phi.sum() - 1.0) < 1e-13
        assert np.abs(phi @ xk - X).max() < 1e-12
        a = rng.standard_normal()
        G = rng.standard_normal(3)
        field = a + xk @ G
        fit = psi.T @ field  # (4,): value at X, then gradient
        assert abs(fit[0] - (a + X @ G)) < 1e-11
        assert np.abs(fit[1:] - G).max() < 1e-11


def test_mls_marker_on_node_closed_form(paper_const):
    """A marker on a node: only the node (r = 0) and its 6 face neighbours
    (r = 1/1.3) are inside the support; by symmetry the fit is the weighted
    mean, phi_centre = 1/(1 + 6 W1), phi_face = W1/(1 + 6 W1)."""
    rw, alpha = paper_const["mls_support_rw"], paper_const["mls_alpha"]
    W1 = math.exp(-((1.0 / rw) / alpha) ** 2)
    base, psi = oracle.mls_point(np.array([5.0, -3.0, 7.0]))
    assert list(base) == [5, -3, 7]
    phi = psi[:, 0]
    assert abs(phi[13] - 1.0 / (1.0 + 6.0 * W1)) < 1e-15
    for k in (4, 10, 12, 14, 16, 22):
        assert abs(phi[k] - W1 / (1.0 + 6.0 * W1)) < 1e-15
    others = [k for k in range(27) if k not in (4, 10, 12, 13, 14, 16, 22)]
    assert np.abs(phi[others]).max() == 0.0


def test_mls_support_cutoff(paper_const):
    """Nodes farther than r_w from the marker get no weight (Eq. intKernel);
    nodes inside get W > 0; 27 candidate nodes per marker."""
    rng = np.random.default_rng(3)
    rw = paper_const["mls_support_rw"]
    for _ in range(200):
        X = rng.uniform(0, 10, 3)
        base, psi = oracle.mls_point(X)
        assert psi.shape[0] == int(paper_const["mls_points"])
        dist = np.linalg.norm(_nodes(base) - X[None, :], axis=1)
        outside = dist > rw * (1 + 1e-12)
        inside = dist < rw * (1 - 1e-12)
        assert np.abs(psi[outside]).max(initial=0.0) == 0.0
        assert inside.sum() >= 4


def test_mls_nearest_block_choice_irrelevant_at_ties():
    """At a half-integer coordinate the support block is ambiguous; nodes that
    differ between the two choices lie beyond r_w, so the weights agree."""
    X = np.array([3.5, 2.25, 1.75])
    Xm = X.copy()
    Xm[0] = np.nextafter(3.5, 0.0)
    b1, p1 = oracle.mls_point(X)
    b2, p2 = oracle.mls_point(Xm)
    assert b1[0] == 4 and b2[0] == 3
    n1, n2 = _nodes(b1), _nodes(b2)
    w1 = {tuple(n): p1[k, 0] for k, n in enumerate(n1) if p1[k, 0] != 0.0}
    w2 = {tuple(n): p2[k, 0] for k, n in enumerate(n2) if p2[k, 0] != 0.0}
    assert set(w1) == set(w2)
    assert max(abs(w1[k] - w2[k]) for k in w1) < 1e-12


def _capsule_sim(n=24, level=2, radius=4.0, tau=0.8, shear=2e-3, Ca=0.1, steps=3, periodic=True):
    c = (n - 1) / 2.0
    v, f = W.icosphere(level, radius, (c + 0.23, c - 0.31, c + 0.17))
    v = W.perturb(v, 0.05, seed=9)
    bc = (0, 0, 0) if periodic else (0, 0, 1)
    U = shear * (n - 1) / 2
    s = oracle.Sim((n, n, n), tau, bc=bc, wall_u=W.shear_walls(U).ravel())
    u0 = W.couette_profile((n, n, n), U)
    s.set_fields(np.ones(n ** 3), u0)
    ks0 = W.ks0_from_capillary(Ca, tau, shear, radius)
    s.add_body(v, f, ks0=ks0, Eb=0.01, kv=10.0, ref_radius=radius)
    assert s.step(steps) == 0
    return s, f


def test_spreading_conserves_force_and_is_adjoint():
    """Eq. (bodyforce) with c_l = A_l: the Eulerian total equals
    sum_l A_l F_l, and spreading is the adjoint of interpolation:
    sum_x f_ib . u* = sum_l A_l F_l . U_l (same shape functions)."""
    s, tris = _capsule_sim()
    fib = s.fib()
    _, us = s.predictor()
    Xn, Ub, Fl = s.markers(0)
    # the last step spread from the positions reached after the step before
    # it; an identical run stopped one step earlier returns them
    s2, _ = _capsule_sim(steps=2)
    Xprev, _, _ = s2.markers(0)
    U = Ub - Fl
    Av = np.zeros(len(Xprev))
    a, b, c = Xprev[tris[:, 0]], Xprev[tris[:, 1]], Xprev[tris[:, 2]]
    At = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    for q in range(3):
        np.add.at(Av, tris[:, q], At / 3.0)
    total_lag = (Av[:, None] * Fl).sum(0)
    assert np.abs(fib.sum(0) - total_lag).max() < 1e-13 * max(1.0, np.abs(total_lag).max())
    lhs = (fib * us).sum()
    rhs = (Av[:, None] * Fl * U).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(rhs) + 1e-20


def test_fluid_momentum_gain_equals_spread_force():
    """Fully periodic box with a capsule: per step the fluid momentum grows by
    exactly the spread force sum_x f_ib."""
    s, _ = _capsule_sim(steps=2)
    e, _ = oracle.lattice()
    p0 = (s.populations() @ e).sum(0)
    assert s.step(1) == 0
    p1 = (s.populations() @ e).sum(0)
    # round-off of summing ~1.4e4 cell momenta of size ~1e-2
    assert np.abs(p1 - p0 - s.fib().sum(0)).max() < 1e-12
