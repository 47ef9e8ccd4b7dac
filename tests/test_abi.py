"""CPU checks of the C-ABI library (no GPU needed): it builds for sm_103a,
loads, exports every function that include/mr_lbm.h declares, and its
host-side flattened weights (Eq. PredictionWithMatrixNew) agree with the
matrix of Eq. PredictionWithMatrix and with the CPU oracle's reconstruction.
"""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_02903_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mr_lbm_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_names(lib):
    lib.mr_lbm_strerror.restype = ctypes.c_char_p
    assert lib.mr_lbm_strerror(0) == b"MR_OK"
    assert b"capacity" in lib.mr_lbm_strerror(4)


def test_create_rejects_bad_config(lib):
    from paper_2103_02903_gb300 import binding, workloads
    cfg, _ = workloads.advection_1d(max_level=6)
    cfg["eps"] = -1.0
    c = binding.make_config(cfg)
    h = ctypes.c_void_p()
    assert binding.library().mr_lbm_create(ctypes.byref(c), None, ctypes.byref(h)) == 1
    cfg, _ = workloads.advection_1d(max_level=6)
    cfg["bc"] = ["periodic", "copy", "periodic", "periodic", "periodic", "periodic"]
    c = binding.make_config(cfg)
    assert binding.library().mr_lbm_create(ctypes.byref(c), None, ctypes.byref(h)) == 1


def _bad(name):
    """One invalid configuration per rule of mr_lbm_create's validation."""
    from paper_2103_02903_gb300 import workloads as W
    cases = {
        "negative_eps": (W.advection_1d, dict(max_level=6), dict(eps=-1.0)),
        "lambda_zero": (W.advection_1d, dict(max_level=6), dict(lambda_=0.0)),
        "relaxation_above_2": (W.advection_1d, dict(max_level=6), dict(s=[2.5] + [0.0] * 15)),
        "mu_bar_negative": (W.advection_1d, dict(max_level=6), dict(mu_bar=-1)),
        "mu_bar_above_order": (W.advection_1d, dict(max_level=6), dict(mu_bar=4)),
        "min_level_below_2": (W.advection_1d, dict(max_level=6), dict(min_level=1)),
        "max_below_min": (W.advection_1d, dict(max_level=6), dict(min_level=5, max_level=4)),
        "max_level_16": (W.advection_1d, dict(max_level=6), dict(max_level=16)),
        "prediction_s4": (W.advection_1d, dict(max_level=6), dict(pred_s=4)),
        "mu_bar_above_order_s2": (W.advection_1d, dict(max_level=6), dict(pred_s=2, mu_bar=6)),
        "half_periodic_axis": (W.advection_1d, dict(max_level=6),
                               dict(bc=["periodic", "copy"] + ["periodic"] * 4)),
        "obstacle_not_d2q9": (W.euler_2d, dict(max_level=5), dict(obstacle=1)),
        "moving_wall_not_d2q9": (W.euler_2d, dict(max_level=5), dict(bc=["bounce_back_velocity"] * 6)),
        "printed_sign_d2q9": (W.ns_obstacle_2d, dict(max_level=5), dict(cross_sign=-1)),
        "exact_collision_fp16": (W.euler_2d, dict(max_level=5), dict(exact_collision=1, precision="fp16")),
        "exact_collision_3d": (W.advection_3d, dict(max_level=4), dict(exact_collision=1)),
        "d3q6_level_11": (W.advection_3d, dict(max_level=4), dict(max_level=11)),
        "d3q6_dense_space": (W.advection_3d, dict(max_level=4), dict(max_level=10)),
        "d2_dense_space": (W.euler_2d, dict(max_level=5), dict(max_level=15)),
        "roots_overflow_codes": (W.euler_2d, dict(max_level=5), dict(roots=[1024, 1024, 1], max_level=12)),
    }
    make, kw, change = cases[name]
    cfg, _ = make(**kw)
    cfg.update(change)
    return cfg


@pytest.mark.parametrize("name", [
    "negative_eps", "lambda_zero", "relaxation_above_2", "mu_bar_negative", "mu_bar_above_order",
    "min_level_below_2",
    "max_below_min", "max_level_16", "prediction_s4",
    "mu_bar_above_order_s2", "half_periodic_axis", "obstacle_not_d2q9",
    "moving_wall_not_d2q9", "printed_sign_d2q9", "exact_collision_fp16", "exact_collision_3d",
    "d3q6_level_11", "d3q6_dense_space", "d2_dense_space", "roots_overflow_codes"])
def test_create_rejects_each_invalid_config(lib, name):
    """Every rule is checked on the host before any device call, so this
    runs without a GPU: MR_EINVAL (1) and a NULL handle."""
    from paper_2103_02903_gb300 import binding
    c = binding.make_config(_bad(name))
    h = ctypes.c_void_p(1)
    assert binding.library().mr_lbm_create(ctypes.byref(c), None, ctypes.byref(h)) == 1
    assert not h.value


def _paper_matrix():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "flattening_matrix_1d.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(Fraction(v)) for v in line.split()])
    return np.array(rows)


@pytest.mark.parametrize("gap", [1, 2, 3, 5])
def test_flattened_weights_match_paper_matrix(lib, gap):
    """Interior weights: R_{k-1} is row 2 (index 1) of M^gap applied to
    f_{k-2..k+1}; R_k is the same row shifted by one cell."""
    from paper_2103_02903_gb300.binding import flattened_weights
    P = np.linalg.matrix_power(_paper_matrix(), gap)
    w = flattened_weights(1, 6, 6 + gap, True, 10)
    r_km1 = np.zeros(5)
    r_km1[0:4] = P[1]            # fine cell 2^g k - 1 from f_{k-2..k+1}
    r_k = np.zeros(5)
    r_k[1:5] = P[1]              # fine cell 2^g (k+1) - 1 from f_{k-1..k+2}
    np.testing.assert_allclose(w[0:5], r_km1 - r_k, rtol=0, atol=1e-15)
    l_k = np.zeros(5)
    l_k[0:4] = P[2]              # fine cell 2^g k from f_{k-2..k+1}
    l_kp1 = np.zeros(5)
    l_kp1[1:5] = P[2]
    np.testing.assert_allclose(w[5:10], l_kp1 - l_k, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2, 13, 14, 15])
@pytest.mark.parametrize("gap", [1, 3])
def test_flattened_weights_match_oracle_near_boundaries(lib, k, gap):
    """With constant extension outside the domain, the weights at the
    boundary slots reproduce the oracle's reconstruction of a uniform level."""
    from oracle import Oracle
    from paper_2103_02903_gb300 import workloads
    from paper_2103_02903_gb300.binding import flattened_weights
    cfg, _ = workloads.burgers_1d(max_level=4 + gap, min_level=2)
    level = 4
    n = 1 << level
    rng = np.random.default_rng(k + 100 * gap)
    f = rng.standard_normal(n)
    o = Oracle(cfg)
    z = np.zeros(n, np.int32)
    o.set_leaves(np.full(n, level, np.int32), np.arange(n, dtype=np.int32), z, z, np.stack([f, f]))
    fine = o.reconstruct(cfg["max_level"])[0]
    w = flattened_weights(1, level, cfg["max_level"], False, k)
    win = np.array([f[k + d] if 0 <= k + d < n else 0.0 for d in range(-2, 3)])
    m = 1 << gap
    r_km1 = fine[m * k - 1] if k > 0 else 0.0
    r_k = fine[m * (k + 1) - 1]
    l_k = fine[m * k]
    l_kp1 = fine[m * (k + 1)] if k + 1 < n else 0.0
    assert abs(w[0:5] @ win - (r_km1 - r_k)) < 1e-13
    assert abs(w[5:10] @ win - (l_kp1 - l_k)) < 1e-13


# ---------------------------------------------------------------------------
# flattened weights of the prediction of half-width s (host only)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("gap", [1, 2, 4])
def test_flattened_weights_s1_are_the_transport_tables(lib, periodic, gap):
    from paper_2103_02903_gb300.binding import flattened_weights, flattened_weights_s
    level = 5
    for k in (0, 1, 2, 9, 29, 30, 31):
        a = flattened_weights(1, level, level + gap, periodic, k)
        b = flattened_weights_s(1, 2, 1, level, level + gap, periodic, k)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("gap", [1, 2, 3])
@pytest.mark.parametrize("periodic", [False, True])
def test_flattened_weights_s_match_oracle(lib, s, gap, periodic):
    """The window weights reproduce, for every cell, the difference of the
    finest edge values that the oracle's reconstruction (with the same s)
    gives from a random uniform level: faces with constant extension, or the
    periodic wrap."""
    from oracle import Oracle
    from paper_2103_02903_gb300 import workloads
    from paper_2103_02903_gb300.binding import flattened_weights_s
    level, w = 5, 2 * s
    if periodic:
        cfg, _ = workloads.advection_1d(max_level=level + gap, min_level=2)
    else:
        cfg, _ = workloads.burgers_1d(max_level=level + gap, min_level=2)
    cfg["pred_s"] = s
    n = 1 << level
    rng = np.random.default_rng(7 * s + gap + 100 * periodic)
    f = rng.standard_normal(n)
    o = Oracle(cfg)
    z = np.zeros(n, np.int32)
    o.set_leaves(np.full(n, level, np.int32), np.arange(n, dtype=np.int32), z, z, np.stack([f, f]))
    fine = o.reconstruct(cfg["max_level"])[0]
    m = 1 << gap
    for k in range(n):
        wts = flattened_weights_s(s, w, 1, level, cfg["max_level"], periodic, k)
        cells = [k + d for d in range(-w, w + 1)]
        if periodic:
            win = np.array([f[c % n] for c in cells])
            r_km1, l_kp1 = fine[(m * k - 1) % (m * n)], fine[(m * (k + 1)) % (m * n)]
        else:
            win = np.array([f[c] if 0 <= c < n else 0.0 for c in cells])
            r_km1 = fine[m * k - 1] if k > 0 else 0.0
            l_kp1 = fine[m * (k + 1)] if k + 1 < n else 0.0
        r_k, l_k = fine[m * (k + 1) - 1], fine[m * k]
        assert abs(wts[: 2 * w + 1] @ win - (r_km1 - r_k)) < 1e-12
        assert abs(wts[2 * w + 1:] @ win - (l_kp1 - l_k)) < 1e-12


@pytest.mark.parametrize("s", [1, 2, 3])
def test_flattened_weights_s_support_and_zero_sum(lib, s):
    """The weights reach exactly 2s cells on either side once the gap is at
    least s (a narrower window is refused), and for an interior cell they sum
    to zero: a constant has no net flux."""
    from paper_2103_02903_gb300.binding import MrError, flattened_weights_s
    for gap in range(s, 9):
        w = flattened_weights_s(s, 2 * s, 1, 6, 6 + gap, True, 10)
        assert w[0] != 0.0 or w[4 * s] != 0.0 or w[4 * s + 1] != 0.0 or w[-1] != 0.0  # window ends
        assert abs(w[: 4 * s + 1].sum()) < 1e-14 and abs(w[4 * s + 1:].sum()) < 1e-14
        with pytest.raises(MrError):
            flattened_weights_s(s, 2 * s - 1, 1, 6, 6 + gap, True, 10)
