"""The benchmark's multi-rank path (one independent replica per rank, whole-job
throughput = summed work / slowest rank's time) on two gloo ranks on CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r did (r+1) * 1e9 interactions and (r+1) * 1e6 particle-steps in (r+1) s
    v, ps, t = bench.aggregate(world, (rank + 1) * 1e9, (rank + 1) * 1e6, float(rank + 1))
    q.put((rank, v, ps, t, bench.allmax(world, 10.0 - rank), bench.allsum(world, 1.5)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, ps, t, mx, sm in out:
        assert t == 2.0                      # slowest rank
        assert v == pytest.approx(3e9 / 2.0)  # (1e9 + 2e9) / 2 s
        assert ps == pytest.approx(3e6 / 2.0)
        assert mx == 10.0 and sm == 3.0


def test_single_rank_is_identity():
    import bench
    v, ps, t = bench.aggregate(1, 5e9, 5e6, 2.0)
    assert (v, ps, t) == (2.5e9, 2.5e6, 2.0)
