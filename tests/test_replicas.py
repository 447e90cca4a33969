"""`bench.py --gpus N` runs N independent replicas (the simulations share nothing, so there is
no collective on the data path).  The one cross-rank step, the max-over-ranks time behind the
whole-job throughput, is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, slowest = bench.replica_throughput(1.0 + rank, 1e6, world)   # rank 1 is the slow one
    q.put((rank, value, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, slowest in got:
        assert slowest == pytest.approx(2.0)            # max over ranks
        assert value == pytest.approx(2 * 1e6 / 2.0 / 1e6)   # all ranks' updates / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    value, slowest = bench.replica_throughput(0.5, 2e6, 1)
    assert slowest == 0.5 and value == pytest.approx(4.0)
