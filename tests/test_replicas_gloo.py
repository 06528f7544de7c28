"""World-size-2 gloo test of the multi-GPU host logic (replicas only): the
barrier, the max over ranks of the timed region, and the whole-job
aggregate, run as two CPU processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1409_2908_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.env() == (world, rank, rank)
        replicas.barrier()
        # rank r "took" 10 * (r + 1) ms for 1000 units
        thr, tmax = replicas.aggregate_throughput(1000.0, 10.0 * (rank + 1))
        out[rank] = (thr, tmax)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slowest time (20 ms) and 2 x 1000 units over it
    for r in range(2):
        thr, tmax = out[r]
        assert tmax == pytest.approx(20.0)
        assert thr == pytest.approx(2000.0 / 0.020)


def test_single_process_defaults():
    from paper_1409_2908_gb300 import replicas
    thr, tmax = replicas.aggregate_throughput(500.0, 5.0)
    assert tmax == 5.0 and thr == pytest.approx(500.0 / 0.005)
