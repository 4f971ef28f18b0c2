"""Host-side logic of the multi-GPU bench path, on CPU with two gloo ranks:
replicas report the slowest rank's time and the whole-job rate."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 2.0 + rank  # rank 1 is slower
    t, value = bench.job_throughput(local, units_per_rank=1000.0, dist=dist, device="cpu")
    q.put((rank, t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in out:
        assert t == 3.0
        assert value == pytest.approx(2 * 1000.0 / 3.0)


def test_job_throughput_single_process():
    import bench
    t, v = bench.job_throughput(4.0, 100.0)
    assert t == 4.0 and v == 25.0


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus, ref_budget = 1, 3, 2, 1.0
    assert bench.run_reference(A()) == 0
