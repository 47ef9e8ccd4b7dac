"""Pins of the oracle's "original adaptive" collision (exact_collision = 1).

Sec. 5.3 states that colliding a leaf's averages (Eq. AdaptiveCollision)
equals colliding the reconstructed finest data and averaging (the right-hand
side of Eq. sourceoferror) when the equilibria are linear, and differs by
O(eps) otherwise; the exact form is the latter.  The pins:

- linear equilibria (D1Q2 advection): both collisions agree to rounding,
  because the reconstruction of a leaf averages back to the leaf
  (Eq. ConsistencyPrediction applied level by level);
- every leaf on the finest level (eps = 0 refines the whole tree): B_{j,k}
  is the leaf itself, so both collisions are the same operation, bit for bit;
- mass: the collision conserves m0 on every finest cell, so the averaged
  leaves conserve the total (periodic Burgers);
- composition: for D1Q2 Burgers the exact step equals the post-transport
  reconstruction (or_reconstruct, pinned elsewhere) collided cell by cell
  with the closed-form D1Q2 collision written out here and averaged over
  each leaf's finest cells;
- nonlinear D2Q9 equilibria on smooth vortices: the two collisions differ
  by far more than rounding (inside coarse leaves the reconstruction varies)
  and by little (the paper's O(eps) difference).  Piecewise-constant data
  would not do: a constant reconstructs exactly, and both collisions agree.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W


def _pair(cfg, u):
    a = Oracle(dict(cfg, exact_collision=1))
    b = Oracle(dict(cfg, exact_collision=0))
    a.init(u)
    b.init(u)
    return a, b


def test_linear_equilibria_exact_equals_leaf_collision():
    cfg, u = W.advection_1d(seed=3, max_level=7)
    cfg["s"][0] = 1.6
    a, b = _pair(cfg, u)
    for _ in range(4):
        a.step(1)
        b.step(1)
        la, fa = a.leaves()[0], a.leaves()[4]
        lb, fb = b.leaves()[0], b.leaves()[4]
        assert np.array_equal(la, lb)
        assert np.max(np.abs(fa - fb)) <= 1e-14 * np.max(np.abs(fb))
    assert np.any(la < cfg["max_level"])  # the pin needs leaves above the finest level


def test_finest_leaves_exact_is_the_leaf_collision():
    cfg, u = W.burgers_1d(seed=4, max_level=6, eps=0.0)
    a, b = _pair(cfg, u)
    for _ in range(3):
        a.step(1)
        b.step(1)
        la, _, _, _, fa = a.leaves()
        lb, _, _, _, fb = b.leaves()
        assert np.all(la == cfg["max_level"]) and np.array_equal(la, lb)
        assert np.array_equal(fa, fb)


def test_exact_collision_conserves_mass():
    cfg, u = W.burgers_1d(seed=5, max_level=8, eps=1e-3)
    cfg["bc"] = ["periodic"] * 6
    cfg["s"][0] = 1.5
    a = Oracle(dict(cfg, exact_collision=1))
    a.init(u)
    J = cfg["max_level"]

    def mass():
        lev, _, _, _, f = a.leaves()
        return float(np.sum(f.sum(axis=0) * 2.0 ** (J - lev)))  # finest cells per leaf

    m0 = mass()
    for _ in range(5):
        a.step(1)
        assert abs(mass() - m0) <= 1e-13 * abs(m0)


def test_exact_collision_composition_burgers():
    cfg, u = W.burgers_1d(seed=6, max_level=7, eps=1e-3)
    s, lam = 1.7, cfg["lambda_"]
    cfg["s"][0] = s
    a, b = _pair(cfg, u)
    for _ in range(2):  # evolve to a non-trivial mesh with both forms in step
        a.step(1)
        b.set_leaves(*a.leaves())
    a.adapt()
    b.set_leaves(*a.leaves())
    b.stream_collide(collide=False)
    fr = b.reconstruct(cfg["max_level"])  # post-transport data on every finest cell
    m0 = fr[0] + fr[1]
    m1 = lam * (fr[0] - fr[1])
    m1 = (1.0 - s) * m1 + s * 0.5 * m0 * m0
    g = np.stack([0.5 * (m0 + m1 / lam), 0.5 * (m0 - m1 / lam)])
    lev, ix, _, _, _ = b.leaves()
    J = cfg["max_level"]
    want = np.zeros((2, len(lev)))
    for n, (l, x) in enumerate(zip(lev, ix)):
        w = 1 << (J - l)
        want[:, n] = g[:, x * w:(x + 1) * w].sum(axis=1) / w
    a.stream_collide(collide=True)
    la, xa, _, _, got = a.leaves()
    assert np.array_equal(la, lev) and np.array_equal(xa, ix)
    assert np.any(lev < J)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_nonlinear_2d_exact_differs_slightly():
    cfg, u = W.vortices_2d(seed=7, max_level=5, eps=1e-3)
    a, b = _pair(cfg, u)
    a.step(1)
    b.step(1)
    la, _, _, _, fa = a.leaves()
    lb, _, _, _, fb = b.leaves()
    assert np.array_equal(la, lb) and np.any(la < cfg["max_level"])
    diff = np.max(np.abs(fa - fb)) / np.max(np.abs(fb))
    assert 1e-10 < diff < 1e-2
