"""D2Q9 (diagonal velocities), the wall with a velocity and the obstacle
penalisation of Sec. 7.2.2 on the CUDA path, against the CPU oracle.

The oracle sums the finest cells of E and A literally; the CUDA path splits
a diagonal velocity into the two axis strips plus four corner cells and
corrects refined neighbours with one-level details.  Leaf sets must agree
exactly, populations within 1e-12 (max-norm relative).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_gpu_parity import _solver, compare, load_oracle_state

pytestmark = pytest.mark.gpu


def _box(seed, bc, max_level=6, eps=1e-4):
    """Vortices in a closed box: every face has the condition `bc`, so
    diagonal populations cross two faces at each corner of the domain."""
    cfg, u = W.vortices_2d(seed=seed, max_level=max_level, eps=eps, bc=bc)
    if bc == "bounce_back_velocity":
        cfg["phys"][0:3] = [1.0, 0.03, -0.02]
    return cfg, u


CASES = [
    ("ns_obstacle J7", lambda s: W.ns_obstacle_2d(seed=s, max_level=7)),
    ("vortices periodic J7", lambda s: W.vortices_2d(seed=s, max_level=7)),
    ("vortices copy J6", lambda s: _box(s, "copy")),
    ("vortices bounce back J6", lambda s: _box(s, "bounce_back")),
    ("vortices anti bounce back J6", lambda s: _box(s, "anti_bounce_back")),
    ("vortices moving wall J6", lambda s: _box(s, "bounce_back_velocity")),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("seed", [0, 1])
def test_d2q9_per_step_from_identical_state(name, make, seed):
    cfg, u = make(seed)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(10):
        load_oracle_state(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s seed %d step %d" % (name, seed, it))


@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_d2q9_trajectory(name, make):
    cfg, u = make(3)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(25):
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s step %d" % (name, it))


def test_d2q9_eps_zero_is_uniform_reference():
    """eps = 0 keeps the full finest mesh: the step is the plain D2Q9 scheme
    on level J (Sec. 3), here with the obstacle and moving walls."""
    cfg, u = W.ns_obstacle_2d(seed=4, max_level=6, eps=0.0)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    gpu.step(6)
    ref.step(6)
    assert gpu.num_leaves() == 2 * 64 * 64
    compare(gpu, ref, cfg, "eps 0")


def test_d2q9_mixed_levels_with_refined_diagonal_neighbours():
    """A mesh built to put refined cells diagonally next to coarse leaves:
    the oracle's leaves after adaptation of a sharp vortex, one step compared
    per level pattern (the leaf set holds every level J_min..J)."""
    cfg, u = W.vortices_2d(seed=5, max_level=7, eps=3e-4, n_vortices=2)
    ref = Oracle(cfg)
    ref.init(u)
    ref.step(3)
    lev = ref.leaves()[0]
    assert len(set(lev.tolist())) >= 4
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(4):
        load_oracle_state(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "mixed levels step %d" % it)


def test_obstacle_relaxes_to_rest_inside_disc():
    """A leaf whose finest-cell centres all lie in the disc (phi = 1) holds
    f^eq(rho0, 0) after the step: zero momentum, density rho0."""
    from test_gpu_parity import gpu_leaves
    cfg, u = W.ns_obstacle_2d(seed=0, max_level=7)
    gpu = _solver(cfg)
    gpu.init(u)
    gpu.step(3)
    J = cfg["max_level"]
    lev, xs, ys, f = gpu_leaves(gpu, cfg)
    cx, cy, r = cfg["phys"][3:6]
    h = 1.0 / (1 << J)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
    full = 0
    for i in range(len(lev)):
        w = 1 << (J - int(lev[i]))
        c = (np.arange(w) + 0.5) * h
        bx, by = np.meshgrid(xs[i] * w * h + c, ys[i] * w * h + c)
        if ((bx - cx) ** 2 + (by - cy) ** 2 <= r * r).all():
            full += 1
            assert abs(float(ex @ f[:, i])) < 1e-15 and abs(float(ey @ f[:, i])) < 1e-15
            assert abs(float(f[:, i].sum()) - cfg["phys"][0]) < 1e-14
    assert full > 0


def test_d2q9_printed_cross_sign_is_rejected():
    from paper_2103_02903_gb300.binding import MrError
    cfg, u = W.vortices_2d(seed=0, max_level=5)
    cfg["cross_sign"] = -1
    with pytest.raises(MrError):
        _solver(cfg)
