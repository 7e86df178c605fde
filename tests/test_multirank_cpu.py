"""The N > 1 path of bench.py (independent replicas, weak scaling) on two
gloo ranks on the CPU: the whole-job time is the slowest rank's, and the
reference arm works and prints on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as d
    d.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    t = bench.slowest_rank_time(1.5 + rank, "cpu")
    q.put((rank, t))
    d.barrier()
    d.destroy_process_group()


def test_slowest_rank_time_is_the_max_over_two_gloo_ranks():
    if not dist.is_available():
        pytest.skip("torch.distributed unavailable")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    assert res == {0: 2.5, 1: 2.5}


def test_single_rank_time_is_the_local_time():
    import bench
    assert bench.slowest_rank_time(3.25) == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    import synth

    def boom(*a, **k):
        raise AssertionError("rank 1 ran the oracle")

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "OraclePool", boom)
    args = bench.argparse.Namespace(steps=2, warmup=1, gpus=2, workload="mid")
    bench.run_reference(args, synth.make_workload("tiny"))
    assert capsys.readouterr().out == ""
