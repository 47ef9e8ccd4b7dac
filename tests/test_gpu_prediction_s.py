"""The prediction of half-width s = 2, 3 on the GPU against the oracle.

Table 1's wider operators (and their tensor products in 2D and 3D, Sec.
4.1) change every part of the step that touches a stencil: the details and
their group norms, the grading (the parent of every tree cell has its
(2s+1)^d neighbourhood in the tree), the ghosts and the transport windows
(2s cells on either side of a leaf, refined cells anywhere in that window
adding the details of their children), the prediction of new leaves and
ghosts, and the reconstruction on a uniform level.  The oracle implements
the same operators literally (pinned in tests/test_oracle_prediction_s.py).

Same bar as for s = 1: leaf sets bit-exact, populations within 1e-12 of
each population field's max norm, per step from the oracle's state (the
decisions must then agree bit for bit) and along independent trajectories
(a decision may differ only within rounding of its threshold, see
test_gpu_fullsize_parity.py), on periodic and copy faces, in 1D, 2D and 3D,
plus the reduced-precision forms, the batch and the refusals.  D2Q9 adds the
diagonal velocities' corner terms over the (4s+1)^2 block around each leaf,
with moving-wall bounce back, the obstacle and the corners of a closed box.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_gpu_fullsize_parity import _check, _load, _solver, _trajectory

pytestmark = pytest.mark.gpu


def _euler_periodic(seed, **kw):
    cfg, u = W.euler_2d(seed=seed, **kw)
    cfg["bc"] = ["periodic"] * 6
    return cfg, u


CASES = [
    ("advection_1d periodic", lambda s: W.advection_1d(seed=s, max_level=8), 30),
    ("burgers_1d copy", lambda s: W.burgers_1d(seed=s, max_level=9), 30),
    ("shallow_water_1d copy", lambda s: W.shallow_water_1d(seed=s, max_level=9), 30),
    ("euler_2d copy", lambda s: W.euler_2d(seed=s, max_level=6), 12),
    ("euler_2d periodic", lambda s: _euler_periodic(s, max_level=6), 12),
    ("advection_3d periodic", lambda s: W.advection_3d(seed=s, max_level=4), 4),
    ("d2q9 vortices periodic", lambda s: W.vortices_2d(seed=s, max_level=6), 10),
    ("d2q9 obstacle, moving walls", lambda s: W.ns_obstacle_2d(seed=s, max_level=6), 10),
    ("d2q9 closed box, bounce back", lambda s: W.vortices_2d(seed=s, max_level=6, bc="bounce_back"), 10),
]


def _cfg(make, seed, s):
    cfg, u = make(seed)
    cfg["pred_s"] = s
    cfg["mu_bar"] = min(cfg["mu_bar"], 2 * s + 1)
    return cfg, u


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_per_step_from_identical_state(name, make, steps, s):
    cfg, u = _cfg(make, 0, s)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    levels = set()
    for it in range(steps):
        if it:
            _load(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        _check(gpu, ref, cfg, "%s s=%d step %d" % (name, s, it))
        levels |= set(ref.leaves()[0].tolist())
    assert len(levels) >= 2, "the mesh should span several levels"


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_trajectory(name, make, steps, s):
    cfg, u = _cfg(make, 1, s)
    restarts, worst = _trajectory(cfg, u, steps, "%s s=%d" % (name, s))
    assert len(restarts) <= 2


@pytest.mark.parametrize("s", [2, 3])
def test_wide_stencil_changes_the_result(s):
    """The same run with s = 1 and with s: the meshes or the fields differ,
    so the wider operator is really in use."""
    cfg, u = W.euler_2d(seed=3, max_level=6)
    a = _solver(cfg)
    a.init(u)
    a.step(6)
    b = _solver(dict(cfg, pred_s=s))
    b.init(u)
    b.step(6)
    pa, pb = a.project(6), b.project(6)
    assert a.num_leaves() != b.num_leaves() or np.abs(pa - pb).max() > 1e-10


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("name,make", [("euler_2d copy", lambda sd: W.euler_2d(seed=sd, max_level=6)),
                                       ("burgers_1d copy", lambda sd: W.burgers_1d(seed=sd, max_level=9)),
                                       ("advection_3d periodic", lambda sd: W.advection_3d(seed=sd, max_level=4))])
def test_project_to_uniform_levels(name, make, s):
    """mr_lbm_project: the reconstruction (projection above the leaves,
    prediction of half-width s below them) on the finest and a middle level."""
    cfg, u = _cfg(make, 4, s)
    ref = Oracle(cfg)
    ref.init(u)
    ref.step(5)
    gpu = _solver(cfg)
    gpu.init(u)
    _load(gpu, ref, cfg)
    J = cfg["max_level"]
    for level in (J, J - 2):
        got, want = gpu.project(level), ref.project(level)
        scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-300)
        assert float((np.abs(got - want) / scale).max()) <= 1e-12, level


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("form,bound", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_reduced_forms(form, bound, s):
    cfg, u = W.euler_2d(seed=5, max_level=6)
    cfg["pred_s"] = s
    ref = Oracle(cfg)
    ref.init(u)
    ref.step(10)
    gpu = _solver(dict(cfg, precision=form))
    gpu.init(u)
    gpu.step(10)
    a, b = gpu.project(6), ref.project(6)
    err = float((np.abs(a - b).sum(axis=1) / np.abs(b).sum(axis=1)).max())
    assert err <= bound


def test_epsilon_zero_full_mesh_s3():
    cfg, u = W.advection_1d(seed=6, max_level=7)
    cfg.update(eps=0.0, pred_s=3)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    ref.step(8)
    gpu.step(8)
    _check(gpu, ref, cfg, "eps 0, s = 3")
    assert gpu.num_leaves() == 1 << 7


def test_batch_mixed_half_widths_equal_each_alone():
    """A batch holding instances of s = 1, 2, 3 (each group of one half-width
    stepped by its own kernels) gives every instance the bits it has alone."""
    from paper_2103_02903_gb300.binding import Batch
    cases = []
    for i, s in enumerate((1, 2, 3, 2)):
        cfg, u = (W.euler_2d if i % 2 == 0 else W.burgers_1d)(seed=20 + i, max_level=6 if i % 2 == 0 else 9)
        cfg["pred_s"] = s
        cases.append((cfg, u))
    b = Batch([c for c, _ in cases])
    for inst, (c, u) in zip(b.instances, cases):
        inst.init(u)
    b.step(5)
    b.synchronize()
    for inst, (c, u) in zip(b.instances, cases):
        solo = _solver(c)
        solo.init(u)
        solo.step(5)
        k1, l1, f1 = inst.get_leaves()
        k2, l2, f2 = solo.get_leaves()
        assert np.array_equal(k1, k2) and np.array_equal(l1, l2) and np.array_equal(f1, f2)
    b.close()


def test_adjoint_refuses_wide_prediction():
    from paper_2103_02903_gb300.binding import MrError
    cfg, u = W.euler_2d(seed=7, max_level=5)
    cfg["pred_s"] = 2
    s = _solver(cfg)
    with pytest.raises(MrError) as ei:
        s.adjoint(u, 4, checkpoint_every=2)
    assert ei.value.status == 1  # MR_EINVAL


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("name,make", [("euler_2d", lambda sd: W.euler_2d(seed=sd, max_level=6)),
                                       ("burgers_1d", lambda sd: W.burgers_1d(seed=sd, max_level=8)),
                                       ("d2q9 obstacle", lambda sd: W.ns_obstacle_2d(seed=sd, max_level=6))])
def test_exact_collision(name, make, s):
    """The original adaptive collision (Eq. sourceoferror) on the
    reconstruction of half-width s, per step from the oracle's state."""
    cfg, u = _cfg(make, 8, s)
    cfg["exact_collision"] = 1
    ref = Oracle(cfg)
    ref.init(u)
    gpu = _solver(cfg)
    gpu.init(u)
    for it in range(6):
        if it:
            _load(gpu, ref, cfg)
        gpu.step(1)
        ref.step(1)
        _check(gpu, ref, cfg, "exact %s s=%d step %d" % (name, s, it))
