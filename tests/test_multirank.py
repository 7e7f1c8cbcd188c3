"""The N-GPU benchmark path is N independent replicas (scenes never exchange data, so there is no
collective on the data path): the only cross-rank step is the whole-job aggregation, checked here
with two gloo ranks on the CPU."""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world_size, port, rank_ms, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    import bench
    value, t_max = bench.job_throughput(1000.0, rank_ms[rank], dist)
    queue.put((rank, value, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_n_times_the_work():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    rank_ms = [100.0, 250.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, rank_ms, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(queue.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, value, t_max in results:
        assert t_max == 250.0                       # the job lasts as long as its slowest rank
        assert value == pytest.approx(2 * 1000.0 / 0.25)


def test_single_process_aggregation_is_the_rank_itself():
    import bench
    value, t = bench.job_throughput(500.0, 200.0)
    assert t == 200.0 and value == pytest.approx(2500.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
