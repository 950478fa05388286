"""The N > 1 path of bench.py on CPU with gloo, world size 2: ranks shard
independent queries (weak scaling, no data-path collective) and only the
timing and the traversed-edge count are reduced: max time, summed edges."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import graphgen as G
    ms, te = bench.reduce_job(10.0 + rank, 1000 * (rank + 1), dist, torch.device("cpu"))
    # each rank draws its own seeded sources (sharded queries)
    g = G.rmat(8, 8, seed=1)
    srcs = bench.make_sources(g, dict(graph="rmat", nsrc=4), rank)
    q.put((rank, ms, te, [int(x) for x in srcs]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for _, ms, te, _ in out:
        assert ms == 11.0 and te == 3000.0
    assert out[0][3] != out[1][3]
