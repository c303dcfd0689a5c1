"""bench.py's multi-rank timing (replicas): max seconds and total units over
ranks, checked with two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    bench.dist_init(world, "gloo")
    t, u = bench.reduce_timing(1.0 + rank, 100.0 * (rank + 1), world)
    bench.barrier(world)
    out.put((rank, t, u))
    dist.destroy_process_group()


def test_reduce_timing_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in res:
        assert t == 2.0 and u == 300.0


def test_reduce_timing_single_rank():
    import bench
    assert bench.reduce_timing(1.5, 7.0, 1) == (1.5, 7.0)
