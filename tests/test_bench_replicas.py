"""The multi-GPU form of the benchmark runs independent replicas (one per GPU,
no data exchange): the reported throughput is the work of all ranks over the
slowest rank's time.  Checked with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    seconds = [2.0, 3.0][rank]
    value, t_max = bench.replica_throughput(world, 6e12, seconds)
    bench._barrier(world)
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, value, t_max in res:
        assert t_max == pytest.approx(3.0)
        assert value == pytest.approx(2 * 6e12 / 3.0 / 1e12)


def test_single_rank_needs_no_process_group():
    import bench

    value, t = bench.replica_throughput(1, 1e12, 0.5)
    assert t == 0.5 and value == pytest.approx(2.0)
