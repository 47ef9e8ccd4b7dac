"""The multi-process path of `bench.py --gpus N` on CPU (gloo, world size 2).

The adaptive step of one instance is not sharded: N ranks run N replicas and
exchange only the final figures, leaf updates summed over the ranks and the
time of the slowest rank.  These tests run that exchange with two gloo
ranks on the host, and the rule of the reference arm under torchrun (rank 0
alone measures; the other ranks exit without work).
"""
import os
import socket
import sys

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2103_02903_gb300.replicas import aggregate
    out = aggregate(100.0 * (rank + 1), 1.0 + 0.5 * rank)
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # updates summed (100 + 200), time of the slowest rank (1.5 s), on every rank
    assert got == {0: (300.0, 1.5), 1: (300.0, 1.5)}


def test_aggregate_without_process_group():
    from paper_2103_02903_gb300.replicas import aggregate
    assert aggregate(5, 2.0) == (5.0, 2.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    args = bench._args()
    assert bench.run_reference(args) == 0
