"""Host logic of the multi-rank benchmark path on CPU with the gloo backend:
each rank advances its own patch (weak scaling, no data-path collective); the
timing is the max over ranks and the value counts every rank's cells.  A rank
that is lost between steps is detected by the others' next collective, which
ends with an error (short process-group timeout) instead of waiting forever."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    m = bench.max_over_ranks(ms)
    q.put((rank, m, bench.whole_job_rate(world, 96 ** 3, 40, m)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] == pytest.approx(2 * 96 ** 3 * 40 / 15e-3)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 10, 4, 2.0) == pytest.approx(10 * 4 / 2e-3)


def _lost_rank_worker(rank, world, port, q):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()  # the message is out before the process vanishes
        os._exit(0)  # lost between steps: no collective in flight, never returns
    try:
        bench.max_over_ranks(10.0)
        q.put((rank, "no error"))
    except Exception as e:  # the collective ends with an error on the host
        q.put((rank, "error: " + type(e).__name__))


def test_lost_rank_ends_the_next_collective_with_an_error():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lost_rank_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert out[1] == "left"
    assert out[0].startswith("error"), out[0]
