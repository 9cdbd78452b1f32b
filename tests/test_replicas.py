"""The multi-rank host logic of bench.py on CPU: two gloo ranks (torchrun-style environment),
barrier, max over ranks of the step time and the whole-job throughput; the reference arm runs
on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo", "cpu")
    reps.barrier()
    seconds = 1.0 + rank          # rank 1 is the slower one
    q.put((rank, reps.max(seconds), reps.throughput(100.0, seconds)))
    reps.close()


def test_two_gloo_ranks_max_time_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, value in got:
        assert t == 2.0                      # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    a = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(a) == 0       # returns at once: no oracle work, no output
