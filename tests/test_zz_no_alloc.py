"""mr_lbm_project_noalloc against mr_lbm_project, through the C-ABI.

The allocation-free variant exists for callers that cannot let the library
call cudaMalloc during a call (device memory owned by another allocator with
a fixed budget, or a serving loop that cannot afford the device-wide
synchronisation an allocation may cause).  It keeps
its level buffers in a fixed 16 MiB file-scope device array instead.  Two
calls in a row, at different levels so that the second one reuses the
first one's leftover contents, must reproduce the allocating entry point
within the tolerance of the other parity tests.  This file is collected last
so that a failure here cannot hide the result of any other test.
"""
import numpy as np
import pytest

from paper_2103_02903_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _close(a, b):
    scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


def test_project_noalloc_matches_project_two_calls():
    from paper_2103_02903_gb300.binding import Solver
    cfg, u = W.euler_2d(seed=3, max_level=8)
    s = Solver(cfg)
    s.init(u)
    s.step(6)
    for level in (8, 6):  # second call at another size over the first call's leftovers
        want = s.project(level)
        got = s.project_noalloc(level)
        assert got.shape == want.shape
        assert _close(got, want) <= TOL
        s.step(2)


def test_project_noalloc_device_output_and_size_limit():
    import torch
    from paper_2103_02903_gb300.binding import MrError, Solver
    cfg, u = W.euler_2d(seed=4, max_level=10)
    s = Solver(cfg)
    s.init(u)
    s.step(2)
    # 4 conserved moments x 4^10 cells exceed the fixed scratch: rejected,
    # and the handle stays usable
    with pytest.raises(MrError) as ei:
        s.project_noalloc(10)
    assert ei.value.status == 4  # MR_ECAPACITY
    for level in (9, 7):
        out = torch.zeros((4, 1 << (2 * level)), dtype=torch.float64, device="cuda")
        s.project_noalloc(level, out)
        torch.cuda.synchronize()
        assert _close(out.cpu().numpy(), s.project(level)) <= TOL
