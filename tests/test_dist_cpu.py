"""Multi-rank host logic of bench.py (barrier, max-over-ranks time, summed work)
with world_size-2 gloo ranks on the CPU."""
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
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      BPP_BENCH_BACKEND="gloo")
    import bench
    r, w = bench.dist_init(world)
    bench.barrier(w)
    mx = bench.allreduce_max(10.0 + r, w)
    sm = bench.allreduce_sum(1.5 * (r + 1), w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, mx, sm))


@pytest.mark.timeout(120)
def test_bench_multirank_helpers_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert res == [(0, 2, 11.0, 4.5), (1, 2, 11.0, 4.5)]
