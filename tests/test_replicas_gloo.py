"""Multi-GPU form of bench.py ("replicas only": independent circuits per
rank, no collective on the data path): the host logic -- disjoint seeds,
max-over-ranks timing, whole-job value -- on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        local_ms = 100.0 + 50.0 * r                   # rank 1 is slower
        mx = bench.job_max_ms(local_ms, dist, "cpu")
        val = bench.job_value(40 * 5, w, mx)
        dist.barrier()
        q.put((r, w, local, bench.replica_seed(r), mx, val))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [x[0] for x in res] == [0, 1]
    assert all(x[1] == 2 for x in res)
    assert res[0][3] != res[1][3]                      # disjoint circuit streams
    assert all(x[4] == 150.0 for x in res)             # max over ranks
    assert all(x[5] == pytest.approx(2 * 200 / 0.150) for x in res)
