"""The multi-GPU form of the benchmark is independent replicas (one per rank,
no data-path collective): only the timings are reduced, by maximum over ranks.
Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    times = bench.max_over_ranks([1.0 + rank, 5.0 - rank], world)
    value = bench.replica_value(100.0, world, times[0])
    out.put((rank, times, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_value_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, value in res:
        assert times == [2.0, 5.0]          # slowest rank per timing
        assert value == pytest.approx(100.0)  # 2 ranks x 100 units / 2 s


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.replica_value(10.0, 1, 2.0) == 5.0
