"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
timed totals are reduced to their maximum over ranks and the whole-job QPS
counts every rank's queries; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        totals = {"mlp": 1.0 + rank, "plain": 3.0 - rank, "_e2e": 0.5 * (rank + 1)}
        red = bench.max_over_ranks(totals, world, torch.device("cpu"))
        qps = bench.weak_scaling_qps({k: v for k, v in red.items() if k != "_e2e"}, world, nq=100, steps=4)
        out.put((rank, red, qps))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, red, qps in res:
        assert red == {"mlp": 2.0, "plain": 3.0, "_e2e": 1.0}
        assert qps["mlp"] == pytest.approx(2 * 100 * 4 / 2.0)
        assert qps["plain"] == pytest.approx(2 * 100 * 4 / 3.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    t = {"a": 1.5, "b": 2.5}
    assert bench.max_over_ranks(t, 1, None) == t
    assert bench.weak_scaling_qps(t, 1, 10, 2) == {"a": 20 / 1.5, "b": 20 / 2.5}


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        nprobe = None
        ref_queries = 8
        steps = 1
        warmup = 3
        config = "B"

    assert bench.run_reference(A(), rank=1) is None
