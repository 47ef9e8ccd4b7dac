"""Degenerate and ragged configurations of the adaptive step on the GPU
against the oracle, with the same bar as the main parity tests (leaf sets
bit-exact, populations within 1e-12 of each population field's max norm).

- J = J_min: a single level, so the mesh cannot adapt (no internal cells,
  no details, no prediction levels) and the step is the uniform scheme on
  that level.
- J = J_min + 1: two levels, the one configuration with adaptation but no
  grading cascade (a graded tree of two levels needs none).
- Ragged root layouts: 3 x 2 roots in 2D (level-l grids of 3 2^l by 2 2^l
  cells), so no level is a power of two in x and the dense chunks, tiles
  and Morton root prefixes do not line up with the domain's edges, with
  copy and with periodic faces (the wrap runs across the root boundaries);
  3 roots in 1D; 2 x 1 x 1 roots in 3D (periodic), the 3-way codes with a
  root prefix.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
import test_gpu_3d as T3
from test_gpu_parity import compare as compare_12, load_oracle_state as load_12

pytestmark = pytest.mark.gpu


def _solver(cfg):
    from paper_2103_02903_gb300.binding import Solver
    return Solver(cfg)


def _is_3d(cfg):
    return cfg["scheme"] == "d3q6_advection"


def load_oracle_state(gpu, ref, cfg):
    (T3._load if _is_3d(cfg) else load_12)(gpu, ref, cfg)


def compare(gpu, ref, cfg, what):
    if _is_3d(cfg):
        T3._compare(gpu, ref, cfg, what)
    else:
        compare_12(gpu, ref, cfg, what)


def _euler_ragged(seed, max_level, roots, bc):
    """Riemann quadrants of D2Q4^4 Euler on [0, roots_x / 2] x [0, roots_y / 2]
    (square cells), the four states meeting at a seeded point inside."""
    cfg, _ = W.euler_2d(seed=seed, max_level=max_level, min_level=2)
    cfg["roots"] = [roots[0], roots[1], 1]
    cfg["xmax"] = [0.5 * roots[0], 0.5 * roots[1], 1.0]
    cfg["bc"] = [bc] * 6
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    st = W.euler_quadrant_states(rng, cfg["phys"][0], cfg["lambda_"])
    cx, cy = rng.uniform(0.3, 0.7) * cfg["xmax"][0], rng.uniform(0.3, 0.7) * cfg["xmax"][1]
    X, Y = W.cell_centres(cfg)
    quad = np.where(X > cx, np.where(Y > cy, 0, 3), np.where(Y > cy, 1, 2))
    rho, u, v, p = np.array(st)[quad].T
    g = cfg["phys"][0]
    E = p / (g - 1.0) + 0.5 * rho * (u * u + v * v)
    return cfg, np.stack([rho, rho * u, rho * v, E]).astype(np.float64)


def _advection_1d_roots3(seed, max_level):
    """D1Q2 advection on [-3, 3] split into 3 roots (3 2^l cells on level l)."""
    cfg, _ = W.advection_1d(seed=seed, max_level=max_level)
    cfg["roots"] = [3, 1, 1]
    c = np.random.Generator(np.random.PCG64(2000 + seed)).uniform(-2.5, 2.5)
    (x,) = W.cell_centres(cfg)
    u = ((x >= -1.0) & (x <= 1.0)).astype(np.float64) + np.exp(-((x - c) / 0.2) ** 2)
    return cfg, u[None, :].copy()


def _advection_3d_roots2(seed, max_level):
    """D3Q6 ball advection on the periodic box [-0.5, 1.5] x [-0.5, 0.5]^2
    (2 x 1 x 1 roots), the ball centred in the second root."""
    cfg, _ = W.advection_3d(seed=seed, max_level=max_level)
    cfg["roots"] = [2, 1, 1]
    cfg["xmax"] = [1.5, 0.5, 0.5]
    c = np.random.Generator(np.random.PCG64(3000 + seed)).uniform(-0.05, 0.05, 3) + np.array([1.0, 0.0, 0.0])
    X, Y, Z = W.cell_centres(cfg)
    u = (((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) <= 0.15 ** 2).astype(np.float64)
    return cfg, u[None, :]


CASES = {
    "advection_1d_roots_3": lambda s: _advection_1d_roots3(s, 6),
    "advection_3d_roots_2x1x1": lambda s: _advection_3d_roots2(s, 5),
    "advection_1d_single_level": lambda s: W.advection_1d(seed=s, max_level=6, min_level=6),
    "euler_2d_single_level": lambda s: W.euler_2d(seed=s, max_level=5, min_level=5),
    "burgers_1d_two_levels": lambda s: W.burgers_1d(seed=s, max_level=5, min_level=4),
    "euler_2d_two_levels": lambda s: W.euler_2d(seed=s, max_level=5, min_level=4),
    "vortices_2d_two_levels": lambda s: W.vortices_2d(seed=s, max_level=5, min_level=4, eps=1e-4),
    "euler_2d_roots_3x2_copy": lambda s: _euler_ragged(s, 5, (3, 2), "copy"),
    "euler_2d_roots_3x2_periodic": lambda s: _euler_ragged(s, 5, (3, 2), "periodic"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_per_step_from_identical_state(name):
    cfg, u = CASES[name](0)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(6):
        load_oracle_state(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s step %d" % (name, it))
    levels = set(ref.leaves()[0].tolist())
    if cfg["min_level"] == cfg["max_level"]:
        assert levels == {cfg["max_level"]}
    gpu.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_trajectory(name):
    cfg, u = CASES[name](1)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(12):
        gpu.step(1)
        ref.step(1)
        compare(gpu, ref, cfg, "%s trajectory step %d" % (name, it))
    gpu.close()
