"""The multi-GPU form is replicas only (independent problems per rank, no
collective on the data path): the job's time is the slowest rank's and its
throughput sums all ranks' solves.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e = bench.slowest_replica(dist, 100.0 + 50.0 * rank, 300.0 - 10.0 * rank, "cpu")
        q.put((rank, t, e, bench.job_throughput(8, 5, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, e, v in out:
        assert t == 150.0 and e == 300.0  # max over ranks
        assert abs(v - 8 * 5 * 2 / 0.150) < 1e-9
