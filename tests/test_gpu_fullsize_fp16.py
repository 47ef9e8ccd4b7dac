"""The configuration the benchmark times, at its full size: D2Q4^4 Euler on
the Riemann quadrants, J = 10 (1024^2 finest cells), FP32 arithmetic with
FP16 storage, one instance stepped through the C-ABI as `bench.py` steps it.

The oracle follows the first steps (FP64, from the same initial condition):
the conserved moments on the finest level stay within the FP16 form's L1
bound and the leaf counts agree.  The benchmark's later steps are beyond the
oracle's reach in seconds, so after them the test checks what holds at any
size: the leaves are finite, they partition the domain (no leaf is an
ancestor of another and their volumes add up to the domain's), every level
lies in [J_min, J], and the tree is graded (every tree cell above J_min has
the 3^d neighbourhood of its parent in the tree: the grading of Sec. 4.4
that the s = 1 prediction stencil needs).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W

pytestmark = pytest.mark.gpu

J = 10


def _l1(a, b):
    return float((np.abs(a - b).sum(axis=1) / np.abs(b).sum(axis=1)).max())


def _key(l, x, y):
    return (np.asarray(l, np.int64) << 44) | (np.asarray(y, np.int64) << 22) | np.asarray(x, np.int64)


def check_mesh(cfg, lev, x, y):
    J = cfg["max_level"]
    Jmin = cfg["min_level"]
    roots = cfg.get("roots", [1, 1, 1])
    periodic = [cfg["bc"][0] == "periodic", cfg["bc"][2] == "periodic"]
    lev = lev.astype(np.int64)
    assert lev.min() >= Jmin and lev.max() <= J
    # volumes in finest cells add up to the domain
    assert int((np.int64(1) << (2 * (J - lev))).sum()) == roots[0] * roots[1] * (1 << (2 * J))
    # tree = leaves and all their ancestors; no leaf is a strict ancestor of another
    leaves = np.unique(_key(lev, x, y))
    assert len(leaves) == len(lev)
    anc = [_key(a, x[lev > a] >> (lev[lev > a] - a), y[lev > a] >> (lev[lev > a] - a)) for a in range(Jmin, J)]
    anc = np.unique(np.concatenate(anc))
    assert not np.isin(leaves, anc).any(), "a leaf lies inside another leaf"
    tree = np.union1d(leaves, anc)
    # grading: the parent's 3x3 neighbourhood of every tree cell above J_min
    tl = (tree >> 44).astype(np.int64)
    ty = ((tree >> 22) & ((1 << 22) - 1)).astype(np.int64)
    tx = (tree & ((1 << 22) - 1)).astype(np.int64)
    sel = tl > Jmin
    pl, px, py = tl[sel] - 1, tx[sel] >> 1, ty[sel] >> 1
    nx_l = roots[0] << pl
    ny_l = roots[1] << pl
    missing = 0
    for ob in (-1, 0, 1):
        for oa in (-1, 0, 1):
            qx, qy = px + oa, py + ob
            keep = np.ones(len(qx), bool)
            if periodic[0]:
                qx = np.mod(qx, nx_l)
            else:
                keep &= (qx >= 0) & (qx < nx_l)
            if periodic[1]:
                qy = np.mod(qy, ny_l)
            else:
                keep &= (qy >= 0) & (qy < ny_l)
            missing += int((~np.isin(_key(pl[keep], qx[keep], qy[keep]), tree)).sum())
    assert missing == 0, "%d parent neighbourhood cells missing: the tree is not graded" % missing


def test_bench_configuration_full_size():
    from paper_2103_02903_gb300.binding import Solver, decode_keys
    cfg, u = W.euler_2d(seed=0, max_level=J)
    ref = Oracle(cfg)
    ref.init(u)
    gpu = Solver(dict(cfg, precision="fp16"))
    gpu.init(u)
    for it in range(3):
        ref.step(1)
        gpu.step(1)
        err = _l1(gpu.project(J), ref.project(J))
        ng, no = gpu.num_leaves(), ref.num_leaves()
        assert err <= 1e-3, "step %d: L1 distance %.3e to the FP64 oracle" % (it, err)
        assert abs(ng - no) <= 0.01 * no, "step %d: %d leaves, oracle %d" % (it, ng, no)
    for n in (100, 1010):  # the benchmark's warm-up and timed steps: 10 + 1000
        gpu.step(n - gpu.counters()[1])
        keys, lev, f = gpu.get_leaves()
        assert np.isfinite(f).all()
        x, y = decode_keys(cfg, lev, keys)[:2]
        check_mesh(cfg, lev, np.asarray(x, np.int64), np.asarray(y, np.int64))
    gpu.close()
