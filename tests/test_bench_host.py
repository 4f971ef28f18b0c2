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


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with every key of the benchmark contract."""
    import json

    import bench
    monkeypatch.setenv("RANK", "0")

    class A:
        steps, warmup, gpus, ref_budget = 1, 3, 1, 0.2
    assert bench.run_reference(A()) in (0, None)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
