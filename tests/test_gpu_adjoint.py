"""Adjoint of the adaptive time step (mr_lbm_adjoint) against central finite
differences, with the mesh of every step frozen.

The adjoint differentiates the map "initial field, relaxation rates ->
functional" along the forward pass's meshes.  A finite difference of the
full adaptive run equals it as long as the perturbation flips no
keep / refine decision, which the tests check by comparing the final leaf
sets of the perturbed runs.  Tolerance: 1e-5 relative (FP64), the bar the
adjoint is built to, plus the rounding floor of the central difference
itself, about 1e-16 |J| / h (h = 1e-7 for the field, relative to its scale,
1e-5 for the rates, which are O(1)).
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _solver(cfg):
    from paper_2103_02903_gb300.binding import Solver
    return Solver(cfg)


def _run(cfg, u, nsteps, K, functional, grads=True):
    s = _solver(cfg)
    out = s.adjoint(u, nsteps, K, functional, gradients=grads)
    keys, lev, _ = s.get_leaves()
    s.close()
    return out, (keys, lev)


def _floor(J, h):
    """Rounding floor of a central difference of J with step h."""
    return 1e-15 * abs(J) / h


def _smooth_direction(cfg, u, seed):
    """A smooth perturbation of every conserved moment (low modes only, so
    that the details, and the mesh, barely move)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = W.cell_centres(cfg)
    L = [cfg["xmax"][a] - cfg["xmin"][a] for a in range(len(X))]
    v = np.zeros_like(u)
    for k in range(u.shape[0]):
        for m in range(1, 4):
            ph = rng.uniform(0, 2 * math.pi, len(X))
            term = rng.standard_normal()
            for a in range(len(X)):
                term = term * np.sin(2 * math.pi * m * (X[a] - cfg["xmin"][a]) / L[a] + ph[a])
            v[k] += term
        v[k] *= np.abs(u[k]).max() + 1e-3
    return v


def _fd_check(cfg, u, nsteps, K, functional, seed=0, rates=(), h=1e-7, hr=1e-5):
    (J, gu, gs), mesh0 = _run(cfg, u, nsteps, K, functional)
    v = _smooth_direction(cfg, u, seed)
    (Jp, _, _), mp = _run(cfg, u + h * v, nsteps, K, functional, grads=False)
    (Jm, _, _), mm = _run(cfg, u - h * v, nsteps, K, functional, grads=False)
    assert np.array_equal(mp[0], mm[0]) and np.array_equal(mp[1], mm[1]), "perturbation changed the mesh"
    fd = (Jp - Jm) / (2 * h)
    ad = float((gu * v).sum())
    assert abs(ad - fd) <= TOL * abs(fd) + _floor(J, h), "initial field: adjoint %.12e vs FD %.12e" % (ad, fd)
    for r in rates:
        cp, cm = dict(cfg), dict(cfg)
        cp["s"] = list(cfg["s"])
        cm["s"] = list(cfg["s"])
        cp["s"][r] += hr
        cm["s"][r] -= hr
        (Jp, _, _), mp = _run(cp, u, nsteps, K, functional, grads=False)
        (Jm, _, _), mm = _run(cm, u, nsteps, K, functional, grads=False)
        assert np.array_equal(mp[0], mm[0]), "rate perturbation changed the mesh"
        fd = (Jp - Jm) / (2 * hr)
        assert abs(gs[r] - fd) <= TOL * abs(fd) + _floor(J, hr), "s[%d]: adjoint %.12e vs FD %.12e" % (r, gs[r], fd)
    return J, gu, gs


def test_adjoint_d1q2_advection():
    cfg, u = W.advection_1d(seed=0, max_level=7)
    _fd_check(cfg, u, 20, 7, "ke_sum", rates=(0,))


def test_adjoint_d1q3_shallow_water_copy_boundaries():
    cfg, u = W.shallow_water_1d(seed=1, max_level=8)
    _fd_check(cfg, u, 25, 10, "ke_final", rates=(0,))


def test_adjoint_d2q4x4_euler():
    cfg, u = W.euler_2d(seed=2, max_level=6)
    _fd_check(cfg, u, 12, 5, "ke_sum", rates=(0, 5))


def test_adjoint_d2q9_obstacle_moving_walls():
    """The obstacle flow (penalisation, moving-wall bounce back, copy
    outlet) with the gradients the obstacle set-up asks for: the initial
    field and both relaxation rates."""
    cfg, u = W.ns_obstacle_2d(seed=3, max_level=6)
    _fd_check(cfg, u, 30, 10, "ke_sum", rates=(0, 1))


def test_adjoint_d2q9_obstacle_J9_rates_two_segments():
    """The obstacle configuration at J = 9 (1024 x 512 finest cells), 60
    steps with a checkpoint every 30 (two replayed segments): the gradients
    with respect to both relaxation rates against central differences.

    The adjoint differentiates along the forward pass's meshes; a finite
    difference equals it only if no keep / refine decision flips between
    the two perturbed runs at any step.  Measured on GB300 at this size,
    perturbing the initial field along a smooth direction flips decisions
    somewhere in the run for every step h from 1e-6 down to 1e-8 (the
    differences scatter by 0.5 % to 46 % about the adjoint, even where the
    final meshes agree), so the initial-field gradient is checked on the
    smaller cases above.  The rates move the solution smoothly: at h = 1e-5
    both differences agree with the adjoint to about 1e-6."""
    cfg, u = W.ns_obstacle_2d(seed=5, max_level=9)
    nsteps, K = 60, 30
    (J, gu, gs), _ = _run(cfg, u, nsteps, K, "ke_sum")
    assert np.isfinite(gu).all()
    hr = 1e-5
    for r in (0, 1):
        cp, cm = dict(cfg), dict(cfg)
        cp["s"], cm["s"] = list(cfg["s"]), list(cfg["s"])
        cp["s"][r] += hr
        cm["s"][r] -= hr
        (Jp, _, _), mp = _run(cp, u, nsteps, K, "ke_sum", grads=False)
        (Jm, _, _), mm = _run(cm, u, nsteps, K, "ke_sum", grads=False)
        assert np.array_equal(mp[0], mm[0]) and np.array_equal(mp[1], mm[1]), "rate perturbation changed the mesh"
        fd = (Jp - Jm) / (2 * hr)
        assert abs(gs[r] - fd) <= TOL * abs(fd) + _floor(J, hr), "s[%d]: adjoint %.12e vs FD %.12e" % (r, gs[r], fd)


def test_adjoint_d2q9_closed_box_bounce_back():
    cfg, u = W.vortices_2d(seed=4, max_level=6, bc="bounce_back")
    _fd_check(cfg, u, 20, 6, "ke_sum", rates=(1,))


def _meshes(cfg, u, nsteps):
    s = _solver(cfg)
    s.init(u)
    out = []
    for _ in range(nsteps):
        s.step(1)
        k, l, _ = s.get_leaves()
        out.append((k, l))
    s.close()
    return out


def test_adjoint_perturbation_amplitudes_obstacle_J7():
    """dJ/da_m of the obstacle set-up: the initial y-momentum is
    1e-3 u0 sum_m a_m sin(m pi y) sin(m pi x / 2) (rho = 1), so
    dJ/da_m = <dJ/d(rho v), 1e-3 u0 sin(m pi y) sin(m pi x / 2)>; checked
    against central differences of a_m, 200 steps, checkpoints every 100.
    dJ/da_m is ~1e-6 J here (the base flow is along x), so the difference
    needs a large step: the largest h of 1e-3, 3e-4, 1e-4 whose perturbed
    runs keep every step's mesh is used, and the tolerance carries the
    rounding floor measured for this J (1e-14 J / h)."""
    cfg, u = W.ns_obstacle_2d(seed=5, max_level=7)
    X, Y = W.cell_centres(cfg)
    N = 200
    (J, gu, gs), _ = _run(cfg, u, N, 100, "ke_sum")
    u0 = cfg["phys"][1]
    for m in (1, 3):
        phi = 1e-3 * u0 * np.sin(m * math.pi * Y) * np.sin(m * math.pi * X / 2.0)
        ad = float((gu[2] * phi).sum())
        for h in (1e-3, 3e-4, 1e-4):
            up, um = u.copy(), u.copy()
            up[2] += h * phi
            um[2] -= h * phi
            mp, mm = _meshes(cfg, up, N), _meshes(cfg, um, N)
            if all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for a, b in zip(mp, mm)):
                break
        else:
            pytest.fail("a_%d: every step size changed a mesh decision" % m)
        (Jp, _, _), _ = _run(cfg, up, N, 100, "ke_sum", grads=False)
        (Jm, _, _), _ = _run(cfg, um, N, 100, "ke_sum", grads=False)
        fd = (Jp - Jm) / (2 * h)
        assert abs(ad - fd) <= TOL * abs(fd) + 1e-14 * abs(J) / h, "a_%d: adjoint %.12e vs FD %.12e (h %g)" % (
            m, ad, fd, h)


def test_functional_value_matches_oracle():
    """J of the forward pass against the oracle's trajectory (the same sum
    written out over the oracle's leaves)."""
    cfg, u = W.ns_obstacle_2d(seed=6, max_level=6)
    (J, _, _), _ = _run(cfg, u, 15, 5, "ke_sum", grads=False)
    ref = Oracle(cfg)
    ref.init(u)
    dx = (cfg["xmax"][0] - cfg["xmin"][0]) / (cfg["roots"][0] << cfg["max_level"])
    lam = cfg["lambda_"]
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
    Jr = 0.0
    for _ in range(15):
        ref.step(1)
        lev, ix, iy, iz, f = ref.leaves()
        rho = f.sum(axis=0)
        qx, qy = lam * (ex @ f), lam * (ey @ f)
        vol = dx * dx * 4.0 ** (cfg["max_level"] - lev)
        Jr += float((vol * 0.5 * (qx * qx + qy * qy) / rho).sum())
    assert abs(J - Jr) <= 1e-11 * abs(Jr)


def test_autograd_function():
    import torch
    from paper_2103_02903_gb300.autograd import trajectory_functional
    cfg, u = W.euler_2d(seed=7, max_level=5)
    u_t = torch.tensor(u, dtype=torch.float64, device="cuda", requires_grad=True)
    s_t = torch.tensor(cfg["s"], dtype=torch.float64, requires_grad=True)
    J = trajectory_functional(u_t, s_t, cfg, 8, 4, "ke_sum")
    gu, gs = torch.autograd.grad(2.0 * J, (u_t, s_t))
    (J2, gu2, gs2), _ = _run(cfg, u, 8, 4, "ke_sum")
    assert abs(J.item() - J2) <= 1e-14 * abs(J2)
    np.testing.assert_allclose(gu.cpu().numpy(), 2.0 * gu2, rtol=0, atol=1e-13 * np.abs(gu2).max())
    np.testing.assert_allclose(gs.numpy(), 2.0 * gs2, rtol=0, atol=1e-13 * np.abs(gs2).max())


def test_adjoint_refuses_reduced_precision():
    from paper_2103_02903_gb300.binding import MrError
    cfg, u = W.euler_2d(seed=8, max_level=5)
    cfg["precision"] = "fp16"
    s = _solver(cfg)
    with pytest.raises(MrError):
        s.adjoint(u, 3, 2)
