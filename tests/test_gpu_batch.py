"""Batched stepping (mr_lbm_batch_*): many independent instances advanced by
shared launches must give, instance by instance, exactly what the same
instance gives when stepped alone, and match the CPU oracle."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu


def _mixed(n, seed=0, max_levels=(5, 6, 7), forms=("fp64",)):
    """D2Q9 vortex instances and D2Q4^4 Riemann instances with uneven levels
    and thresholds (the shape of a batched serving load, small sizes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        J = int(rng.choice(max_levels))
        eps = float(rng.choice([1e-3, 1e-4]))
        if i % 2 == 0:
            cfg, u = W.vortices_2d(seed=seed * 1000 + i, max_level=J, eps=eps)
        else:
            cfg, u = W.euler_2d(seed=seed * 1000 + i, max_level=J, eps=eps)
        cfg["precision"] = forms[i % len(forms)]
        out.append((cfg, u))
    return out


def _solo(cfg, u, steps):
    from paper_2103_02903_gb300.binding import Solver
    s = Solver(cfg)
    s.init(u)
    s.step(steps)
    return s.get_leaves()


@pytest.mark.parametrize("forms", [("fp64",), ("fp64", "fp16", "fp32")])
def test_batch_equals_instances_stepped_alone(forms):
    from paper_2103_02903_gb300.binding import Batch
    cases = _mixed(9, seed=1, forms=forms)
    b = Batch([c for c, _ in cases])
    for s, (c, u) in zip(b.instances, cases):
        s.init(u)
    b.step(6)
    b.synchronize()
    for i, (s, (c, u)) in enumerate(zip(b.instances, cases)):
        k1, l1, f1 = s.get_leaves()
        k2, l2, f2 = _solo(c, u, 6)
        assert np.array_equal(l1, l2) and np.array_equal(k1, k2), "instance %d: leaf sets differ" % i
        assert np.array_equal(f1, f2), "instance %d: populations differ" % i
    lu, st = b.counters()
    assert st == 6 and lu > 0
    b.close()


def test_batch_matches_oracle():
    from paper_2103_02903_gb300.binding import Batch
    cases = _mixed(4, seed=2, max_levels=(5, 6))
    b = Batch([c for c, _ in cases])
    refs = []
    for s, (c, u) in zip(b.instances, cases):
        s.init(u)
        r = Oracle(c)
        r.init(u)
        refs.append(r)
    for it in range(5):
        b.step(1)
        for k, (s, r) in enumerate(zip(b.instances, refs)):
            r.step(1)
            compare(s, r, cases[k][0], "batch instance %d step %d" % (k, it))
    b.close()


def test_batch_rules():
    from paper_2103_02903_gb300.binding import Batch, MrError
    cases = _mixed(3, seed=3, max_levels=(5,))
    b = Batch([c for c, _ in cases])
    b.instances[0].init(cases[0][1])
    with pytest.raises(MrError):  # instances 1, 2 not initialised
        b.step(1)
    for s, (c, u) in zip(b.instances[1:], cases[1:]):
        s.init(u)
    b.step(2)
    with pytest.raises(MrError):  # a lent handle cannot step alone
        b.instances[1].step(1)
    b.step(1)
    b.synchronize()
    assert all(s.num_leaves() > 0 for s in b.instances)
    b.close()
