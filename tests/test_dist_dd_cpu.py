"""Multi-process host logic of the decomposition in x4 with world_size-2 gloo
ranks on the CPU: slab ownership and the face messages of one hop, the
point-to-point face exchange (each slab must receive the bottom face of the
slab above and the top face of the slab below, cyclically), and the
cross-process sum of per-slab reductions."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_face_messages_cover_every_slab_once():
    from paper_2111_04457_b300.dd import face_messages, slab_owner
    world, nlocal = 3, 2
    n = world * nlocal
    msgs = face_messages(world, nlocal)
    assert len(msgs) == 2 * n
    got = {(m.dst_slab, m.kind): m for m in msgs}
    assert len(got) == 2 * n and len({m.tag for m in msgs}) == 2 * n
    for g in range(n):
        assert got[(g, "down")].src_slab == (g + 1) % n      # forward buffer: bottom face of the slab above
        assert got[(g, "up")].src_slab == (g - 1) % n        # backward buffer: top face of the slab below
        for kind in ("down", "up"):
            m = got[(g, kind)]
            assert m.src_rank == slab_owner(m.src_slab, nlocal) and m.dst_rank == slab_owner(g, nlocal)


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2111_04457_b300.dd import ProcessReducer, exchange_faces
    nlocal = 2
    mine = [rank * nlocal + k for k in range(nlocal)]
    down = {g: torch.full((3, 5), 10.0 * g + 0.0, dtype=torch.float64) for g in mine}
    up = {g: torch.full((3, 5), 10.0 * g + 1.0, dtype=torch.float64) for g in mine}
    fwd, bwd = exchange_faces(rank, world, nlocal, down, up)
    n = world * nlocal
    ok_faces = all(float(fwd[g][0, 0]) == 10.0 * ((g + 1) % n) and float(bwd[g][0, 0]) == 10.0 * ((g - 1) % n) + 1.0
                   for g in mine) and sorted(fwd) == mine and sorted(bwd) == mine
    # per-slab sums of a global array: rows of the slabs this rank owns
    glob = np.random.default_rng(5).normal(size=(n, 8))
    tot = ProcessReducer()(glob[mine])
    ok_sum = bool(np.allclose(tot, glob.sum(axis=0), rtol=1e-15, atol=1e-15))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ok_faces, ok_sum))


@pytest.mark.timeout(120)
def test_face_exchange_and_reducer_gloo():
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
    assert res == [(0, True, True), (1, True, True)]
