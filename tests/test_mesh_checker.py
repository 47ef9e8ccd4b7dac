"""The mesh-validity check of the full-size GPU test, pinned on the CPU: it
accepts the oracle's adapted meshes (which the oracle's own grading check
accepts) and rejects two planted mistakes, a missing leaf (the volumes no
longer add up) and a coarsened region next to finer leaves (not graded)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_gpu_fullsize_fp16 import check_mesh


@pytest.mark.parametrize("name", ["euler_2d", "vortices_2d", "ns_obstacle_2d"])
def test_check_mesh_on_oracle_meshes(name):
    cfg, u = W.WORKLOADS[name](seed=0, max_level=7)
    o = Oracle(cfg)
    o.init(u)
    o.step(4)
    assert o.graded()
    lev, ix, iy = o.leaves()[:3]
    lev, ix, iy = lev.astype(np.int64), ix.astype(np.int64), iy.astype(np.int64)
    check_mesh(cfg, lev, ix, iy)
    with pytest.raises(AssertionError):
        check_mesh(cfg, lev[1:], ix[1:], iy[1:])
    # replace every leaf inside the level-(J_min+1) cell of the deepest leaf by that cell
    l0 = cfg["min_level"] + 1
    X, Y = ix >> (lev - l0), iy >> (lev - l0)
    k = int(np.argmax(lev))
    inside = (X == X[k]) & (Y == Y[k])
    with pytest.raises(AssertionError, match="not graded"):
        check_mesh(cfg, np.append(lev[~inside], l0), np.append(ix[~inside], X[k]), np.append(iy[~inside], Y[k]))
