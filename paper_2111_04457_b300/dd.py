"""Multi-process side of the decomposition in x4 (the parallelisation of Sec. 2
and Sec. 3.1): which process owns which slab, the face messages of one
decomposed hop, and the cross-process sum of the solver's per-slab
reductions.  Host logic only: the faces are packed and applied by the
library's kernels (bpp_dd_*); with all slabs on one GPU the library copies
them itself, and a reducer built here plugs into
DomainDecomposition.set_reducer.

Slabs are numbered g = 0 .. nslab-1 along x4; process r owns the nlocal
consecutive slabs g = r * nlocal .. r * nlocal + nlocal - 1.  A hop sends, for
every slab g, its bottom face to slab g-1 (there it is the forward face
buffer) and its top face to slab g+1 (the backward face buffer), cyclically.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class FaceMessage:
    kind: str          # "down": bottom face to the slab below; "up": top face to the slab above
    src_slab: int      # global slab index of the sender
    dst_slab: int
    src_rank: int
    dst_rank: int
    tag: int           # unique per (destination slab, kind)


def slab_owner(g: int, nlocal: int) -> int:
    return g // nlocal


def face_messages(world: int, nlocal: int) -> list[FaceMessage]:
    """Every face message of one decomposed hop, in slab order."""
    n = world * nlocal
    out = []
    for g in range(n):
        lo, hi = (g - 1) % n, (g + 1) % n
        out.append(FaceMessage("down", g, lo, slab_owner(g, nlocal), slab_owner(lo, nlocal), 2 * lo))
        out.append(FaceMessage("up", g, hi, slab_owner(g, nlocal), slab_owner(hi, nlocal), 2 * hi + 1))
    return out


def exchange_faces(rank: int, world: int, nlocal: int, down: dict, up: dict, group=None):
    """Runs the face messages of this rank with torch.distributed point-to-point
    calls.  down[g] / up[g]: the packed faces (tensors) of this rank's slabs g.
    Returns (fwd, bwd): fwd[g] = the bottom face of slab g+1, bwd[g] = the top
    face of slab g-1, for this rank's slabs g.  Messages between slabs of the
    same rank are copies."""
    import torch.distributed as dist
    fwd, bwd, reqs = {}, {}, []
    msgs = face_messages(world, nlocal)
    # receives first, then sends (non-blocking), so no ordering can deadlock
    like = next(iter(down.values()))
    for m in msgs:
        if m.dst_rank != rank:
            continue
        if m.src_rank == rank:
            buf = (down if m.kind == "down" else up)[m.src_slab].clone()
        else:
            buf = like.new_empty(like.shape)
            reqs.append(dist.irecv(buf, src=m.src_rank, tag=m.tag, group=group))
        (fwd if m.kind == "down" else bwd)[m.dst_slab] = buf
    for m in msgs:
        if m.src_rank != rank or m.dst_rank == rank:
            continue
        t = down[m.src_slab] if m.kind == "down" else up[m.src_slab]
        reqs.append(dist.isend(t, dst=m.dst_rank, tag=m.tag, group=group))
    for r in reqs:
        r.wait()
    return fwd, bwd


class ProcessReducer:
    """Reducer for DomainDecomposition.set_reducer in a multi-process run:
    sums this process's slabs in slab order, then adds the other processes'
    sums with torch.distributed.all_reduce (float64)."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, parts: np.ndarray) -> np.ndarray:
        import torch
        import torch.distributed as dist
        local = np.zeros(parts.shape[1], dtype=np.float64)
        for k in range(parts.shape[0]):
            local += parts[k]
        t = torch.from_numpy(local)
        if dist.is_available() and dist.is_initialized():
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.numpy()
