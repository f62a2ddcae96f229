"""Replica timing across ranks on CPU with the gloo backend (world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2510_27447_gb300.replicas import whole_job_rate
    # rank r processed (r+1) * 1000 node-steps in (r+1) * 0.5 s
    rate, secs = whole_job_rate((rank + 1) * 1000.0, (rank + 1) * 0.5)
    q.put((rank, rate, secs))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_sums_units_and_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, secs in res:
        assert secs == 1.0                      # max over ranks
        assert rate == pytest.approx(3000.0)    # (1000 + 2000) / 1.0


def test_without_process_group_rate_is_local():
    from paper_2510_27447_gb300.replicas import whole_job_rate
    rate, secs = whole_job_rate(500.0, 0.25)
    assert rate == 2000.0 and secs == 0.25
