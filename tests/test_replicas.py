"""The multi-rank path on CPU: two gloo ranks with different timed regions
report the slower one, and the whole-job rate counts both ranks' work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2508_08965_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    job = replicas.job_time_ms(ms)
    rate = replicas.whole_job_rate(1000, 10, job, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, job, rate))


def test_two_gloo_ranks_report_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job, rate in res:
        assert job == pytest.approx(150.0)
        assert rate == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_process_is_local():
    from paper_2508_08965_gb300 import replicas
    assert replicas.job_time_ms(12.5) == 12.5
