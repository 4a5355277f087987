"""Argmax of a grid split across ranks: the packed 64-bit key of the sharded
layout (cells partitioned over GPUs, one maximum reduction per BOMP
iteration).

Every GPU here runs independent replicas, so no collective runs on the data
path; this is the host-side reduction that a sharded grid would use, tested
with gloo ranks on the CPU. A rank's best cell and score are packed as

    key = bits(score) * 2^32 + (2^32 - 1 - cell)

with bits() the IEEE-754 pattern of a non-negative float32 score (ordered
like the scores), so that the maximum key over the ranks is the largest
score and, among equal scores, the smallest cell (the argmax tie rule).
Keys are non-negative int64; a rank without a candidate contributes -1.
"""
from __future__ import annotations

import numpy as np

NO_CANDIDATE = -1
MAX_CELL = (1 << 32) - 1


def pack_argmax_key(score: float, cell: int) -> int:
    """Key of a (score, cell) candidate: score a finite float32 >= 0, cell < 2^32."""
    s = np.float32(score)
    if not np.isfinite(s) or s < 0:
        raise ValueError("score must be a finite non-negative float32")
    if not 0 <= int(cell) < MAX_CELL:
        raise ValueError("cell must lie in [0, 2^32 - 1)")
    bits = int(np.array(s, dtype=np.float32).view(np.uint32))
    return (bits << 32) | (MAX_CELL - int(cell))


def unpack_argmax_key(key: int):
    """(score, cell) of a key, or None for NO_CANDIDATE."""
    key = int(key)
    if key < 0:
        return None
    score = float(np.array(key >> 32, dtype=np.uint32).view(np.float32))
    return score, MAX_CELL - (key & MAX_CELL)


def local_argmax(scores, cells):
    """Best (score, cell) of a shard: largest score, smallest cell among equal
    scores; None for an empty shard."""
    scores = np.asarray(scores, dtype=np.float32).reshape(-1)
    cells = np.asarray(cells, dtype=np.int64).reshape(-1)
    if scores.size == 0:
        return None
    m = scores.max()
    return float(m), int(cells[scores == m].min())


def allreduce_argmax(best, group=None):
    """Global (score, cell) from each rank's local best (or None), by one
    maximum all-reduce of the packed key (torch.distributed)."""
    import torch
    import torch.distributed as dist
    key = NO_CANDIDATE if best is None else pack_argmax_key(*best)
    t = torch.tensor([key], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return unpack_argmax_key(int(t.item()))
