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


def _small_serving(n=8, seed=3):
    cases = W.serving_batch(seed=seed, n=n, levels=(6, 7), precision="fp16")
    return cases


def test_autotune_leaves_the_batch_as_it_was_and_results_do_not_depend_on_the_schedule():
    """mr_lbm_batch_autotune times candidate schedules from a snapshot of
    every instance and puts the snapshot back: the leaves and the counters
    after the call are those before it.  Schedules change grid sizes only,
    so the tuned batch steps to the same bits as one on the default
    schedule; a batch of the same signature created later starts from the
    cached schedule."""
    from paper_2103_02903_gb300.binding import Batch, MrError
    cases = _small_serving()
    a = Batch([c for c, _ in cases])
    ref = Batch([c for c, _ in cases])
    for bb in (a, ref):
        for inst, (c, u) in zip(bb.instances, cases):
            inst.init(u)
        bb.step(3)
        bb.synchronize()
    before = [inst.get_leaves() for inst in a.instances]
    counts = [inst.counters() for inst in a.instances]
    default = a.schedule()
    ms_fixed, ms_tuned = a.autotune(trial_steps=2)
    assert ms_fixed > 0 and ms_tuned > 0
    after = [inst.get_leaves() for inst in a.instances]
    for x, y in zip(before, after):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
    assert [inst.counters() for inst in a.instances] == counts
    tuned = a.schedule()
    assert len(tuned) == a.parts() and all(len(p) == 7 for p in tuned)
    assert all(1 <= v <= 32 for p in tuned for v in p)
    a.step(4)
    ref.step(4)
    for x, y in zip(a.instances, ref.instances):
        for u, v in zip(x.get_leaves(), y.get_leaves()):
            assert np.array_equal(u, v)
    # the cache: a new batch of the same configurations starts tuned
    c = Batch([c for c, _ in cases])
    assert c.schedule() == tuned
    with pytest.raises(MrError):
        c.set_schedule(0, [0] * 7)
    c.set_schedule(0, default[0])
    assert c.schedule()[0] == default[0]
    for bb in (a, ref, c):
        bb.close()
