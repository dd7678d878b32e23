"""The N > 1 path (replicas) on CPU: two gloo ranks on 127.0.0.1 agree on the
slowest rank's time, the summed work, and every rank's calibration report."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1904_09538_gb300 import replicas
    try:
        t = replicas.job_time(1.0 + rank, dist, "cpu")
        v, tt = replicas.job_throughput(100.0 * (rank + 1), 1.0 + 0.5 * rank, dist, "cpu")
        reps = replicas.gather_reports({"rank": rank, "geo": 0.01 * (rank + 1)}, dist)
        q.put((rank, t, v, tt, reps))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_on_gloo():
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
    for rank, t, v, tt, reps in out:
        assert t == 2.0                       # slowest rank's elapsed time
        assert tt == 1.5 and v == 300.0 / 1.5  # all ranks' work over the slowest time
        assert reps == [{"rank": 0, "geo": 0.01}, {"rank": 1, "geo": 0.02}]


def test_single_process_is_identity():
    from paper_1904_09538_gb300 import replicas
    assert replicas.job_time(3.0, dist, "cpu") == 3.0
    assert replicas.job_throughput(10.0, 2.0, dist, "cpu") == (5.0, 2.0)
    assert replicas.gather_reports({"a": 1}, dist) == [{"a": 1}]
