"""The multi-process (replicas-only) path of bench.py on CPU: two gloo ranks
on 127.0.0.1, as torchrun launches them; no GPU."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [40.0, 55.0][rank]  # rank 1 is the slower replica
    total = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.job_throughput(1e9, world, total)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, total, value))


def test_replicas_time_is_the_slowest_rank_and_value_counts_all_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == 55.0
        assert value == pytest.approx(2 * 1e9 / 0.055)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(Args())  # returns at once, prints nothing
    assert capsys.readouterr().out == ""
