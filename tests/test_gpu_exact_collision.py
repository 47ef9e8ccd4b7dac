"""Parity of the original adaptive collision (exact_collision = 1, Sec. 5.3,
Eq. sourceoferror) on the GPU with the oracle's, through the C-ABI.

Same bar as the leaf collision: leaf sets bit-exact, populations within
1e-12 of each population field's max norm.  Cases: the three 1D schemes,
D2Q4^4 Euler, and D2Q9 both periodic and with the obstacle (penalisation
after the averaged collision), per step from the oracle's state and along
independent trajectories; the refusals (reduced precision, batches, the
adjoint) go through the C-ABI's status codes.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_gpu_parity import compare, load_oracle_state

pytestmark = pytest.mark.gpu

CASES = [
    ("burgers_1d", dict(max_level=9), 20),
    ("shallow_water_1d", dict(max_level=9), 20),
    ("advection_1d", dict(max_level=8), 15),
    ("euler_2d", dict(max_level=6), 12),
    ("vortices_2d", dict(max_level=6, eps=3e-4, n_vortices=2), 12),
    ("ns_obstacle_2d", dict(max_level=6), 12),
]


def _solver(cfg):
    from paper_2103_02903_gb300.binding import Solver
    return Solver(cfg)


def _cfg(name, kw, seed):
    cfg, u = W.WORKLOADS[name](seed=seed, **kw)
    cfg["exact_collision"] = 1
    return cfg, u


@pytest.mark.parametrize("name,kw,steps", CASES)
def test_per_step_from_identical_state(name, kw, steps):
    cfg, u = _cfg(name, kw, 0)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    coarse = False
    for it in range(min(steps, 8)):
        load_oracle_state(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s exact step %d" % (name, it))
        coarse = coarse or bool(np.any(ref.leaves()[0] < cfg["max_level"]))
    assert coarse  # leaves above the finest level, where the two collisions differ


@pytest.mark.parametrize("name,kw,steps", CASES)
def test_trajectory(name, kw, steps):
    cfg, u = _cfg(name, kw, 1)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(steps):
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s exact trajectory step %d" % (name, it))


def test_exact_differs_from_leaf_collision_on_gpu():
    """Nonlinear equilibria on smooth data: the two collisions give fields
    that differ by far more than rounding (the difference the paper calls
    O(eps)), each matched by the oracle above.  Piecewise-constant data would
    not show it: a constant reconstructs exactly."""
    cfg, u = W.vortices_2d(seed=2, max_level=6, eps=1e-3)
    a = _solver(dict(cfg, exact_collision=1))
    b = _solver(dict(cfg, exact_collision=0))
    a.init(u)
    b.init(u)
    a.step(2)
    b.step(2)
    ka, la, fa = a.get_leaves()
    kb, lb, fb = b.get_leaves()
    assert np.array_equal(ka, kb) and np.array_equal(la, lb)
    d = np.abs(fa - fb).max() / np.abs(fb).max()
    assert 1e-10 < d < 1e-2


def test_refusals():
    from paper_2103_02903_gb300.binding import Batch, MrError
    cfg, u = _cfg("euler_2d", dict(max_level=5), 3)
    with pytest.raises(MrError):
        _solver(dict(cfg, precision="fp16"))
    with pytest.raises(MrError):
        Batch([cfg, cfg])
    s = _solver(cfg)
    with pytest.raises(MrError):
        s.adjoint(u, 2, 1)
    s.close()
