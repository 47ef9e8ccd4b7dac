"""D3Q6 advection of a ball (Sec. 7.3, d = 3) on the GPU against the oracle.

The same bar as in 1D and 2D: leaf sets bit-exact (keys are 3-way Morton
codes with a root prefix), populations within 1e-12 of each population
field's max norm, per step from the oracle's state and along independent
trajectories; eps = 0 refines the whole tree; the reduced-precision forms
keep their stated L1 distance to the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _solver(cfg):
    from paper_2103_02903_gb300.binding import Solver
    return Solver(cfg)


def _gpu_leaves(s, cfg):
    from paper_2103_02903_gb300.binding import decode_keys3
    keys, lev, f = s.get_leaves()
    x, y, z = decode_keys3(cfg, lev, keys)
    order = np.lexsort((x, y, z, lev))
    return lev[order].astype(np.int64), x[order], y[order], z[order], f[:, order]


def _load(s, ref, cfg):
    from paper_2103_02903_gb300.binding import encode_keys3
    lev, ix, iy, iz, f = ref.leaves()
    s.set_leaves(encode_keys3(cfg, lev, ix, iy, iz), lev.astype(np.int8), f)


def _compare(s, ref, cfg, what):
    glev, gx, gy, gz, gf = _gpu_leaves(s, cfg)
    lev, ix, iy, iz, f = ref.leaves()
    same = (len(glev) == len(lev) and (glev == lev).all() and (gx == ix).all() and (gy == iy).all()
            and (gz == iz).all())
    if not same:
        pytest.fail("%s: leaf sets differ (gpu %d, oracle %d leaves, oracle margin %.3e)"
                    % (what, len(glev), len(lev), ref.margin()))
    scale = np.maximum(np.abs(f).max(axis=1, keepdims=True), 1e-300)
    err = float((np.abs(gf - f) / scale).max())
    assert err <= TOL, "%s: populations differ by %.3e (max-norm relative)" % (what, err)


@pytest.mark.parametrize("seed", [0, 1])
def test_per_step_from_identical_state(seed):
    cfg, u = W.advection_3d(seed=seed, max_level=5)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    levels = set()
    for it in range(6):
        _load(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        _compare(gpu, ref, cfg, "3d seed %d step %d" % (seed, it))
        levels |= set(ref.leaves()[0].tolist())
    assert len(levels) >= 3  # a multi-level 3D mesh


def test_trajectory():
    cfg, u = W.advection_3d(seed=2, max_level=5)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(10):
        gpu.step(1)
        ref.step(1)
        _compare(gpu, ref, cfg, "3d trajectory step %d" % it)


def test_copy_boundaries_and_mu_zero():
    cfg, u = W.advection_3d(seed=3, max_level=5, mu_bar=0)
    cfg["bc"] = ["copy"] * 6
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(6):
        gpu.step(1)
        ref.step(1)
        _compare(gpu, ref, cfg, "3d copy step %d" % it)


def test_epsilon_zero_full_mesh():
    cfg, u = W.advection_3d(seed=4, max_level=4, eps=0.0)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(4):
        gpu.step(1)
        ref.step(1)
        _compare(gpu, ref, cfg, "3d eps=0 step %d" % it)
    assert (ref.leaves()[0] == cfg["max_level"]).all()


@pytest.mark.parametrize("form,bound", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_reduced_precision_forms(form, bound):
    cfg, u = W.advection_3d(seed=5, max_level=5)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(dict(cfg, precision=form))
    gpu.init(u)
    ref.step(8)
    gpu.step(8)
    J = cfg["max_level"]
    a = gpu.project(J)
    b = ref.project(J)
    l1 = np.abs(a - b).sum() / np.abs(b).sum()
    assert l1 <= bound, "%s: relative L1 distance %.3e" % (form, l1)


def test_refusals():
    from paper_2103_02903_gb300.binding import MrError
    cfg, u = W.advection_3d(seed=6, max_level=4)
    with pytest.raises(MrError):
        _solver(dict(cfg, exact_collision=1))
    with pytest.raises(MrError):
        _solver(dict(cfg, max_level=11))
    s = _solver(cfg)
    with pytest.raises(MrError):
        s.adjoint(u, 2, 1)
    s.close()


def test_batch_of_3d_instances_equals_each_alone():
    """3D instances (several finest levels, both forms) in one batch: every
    instance ends bit for bit where it ends stepped alone."""
    from paper_2103_02903_gb300.binding import Batch
    cases = []
    for i, (J, form) in enumerate([(4, "fp64"), (5, "fp64"), (5, "fp16"), (4, "fp16")]):
        cfg, u = W.advection_3d(seed=10 + i, max_level=J)
        cfg["precision"] = form
        cases.append((cfg, u))
    b = Batch([c for c, _ in cases])
    for s, (c, u) in zip(b.instances, cases):
        s.init(u)
    b.step(5)
    b.synchronize()
    for i, (s, (c, u)) in enumerate(zip(b.instances, cases)):
        alone = _solver(c)
        alone.init(u)
        alone.step(5)
        k1, l1, f1 = s.get_leaves()
        k2, l2, f2 = alone.get_leaves()
        assert np.array_equal(l1, l2) and np.array_equal(k1, k2), "instance %d: leaf sets differ" % i
        assert np.array_equal(f1, f2), "instance %d: populations differ" % i
        alone.close()
    b.close()


def test_capacity_and_input_errors():
    from paper_2103_02903_gb300.binding import MrError, encode_keys3
    cfg, u = W.advection_3d(seed=7, max_level=5)
    s = _solver(dict(cfg, leaf_capacity=200))
    with pytest.raises(MrError) as ei:  # the initial full mesh needs 32^3 leaves
        s.init(u)
        s.synchronize()
    assert ei.value.status == 4  # MR_ECAPACITY, reported at the next synchronising call
    s.close()
    s = _solver(cfg)
    s.init(u)
    keys, lev, f = s.get_leaves()
    bad = keys.copy()
    bad[0] = bad[1]  # two leaves on one cell: not a partition
    with pytest.raises(MrError):
        s.set_leaves(bad, lev, f)
    x = np.array([0, 1]), np.array([0, 0]), np.array([0, 0])
    assert list(encode_keys3(cfg, np.array([5, 5]), *x)) == [0, 1]
    s.close()
