"""Host logic of the multi-rank benchmark on CPU (gloo, world size 2): the
whole-job value sums the units of all ranks and divides by the slowest
rank's time; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed 10 + r units in 2 + 3 r seconds
    units, secs = bench.combine_ranks(2.0 + 3.0 * rank, 10 + rank, "cpu")
    q.put((rank, units, secs))
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, secs in out:
        assert units == 21.0   # 10 + 11
        assert secs == 5.0     # max(2, 5)


def test_combine_ranks_single_process():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(1.5, 7, "cpu") == (7.0, 1.5)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
