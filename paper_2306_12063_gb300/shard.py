"""Frame sharding across GPUs.  Frames are independent (every codeword is
decoded on its own), so ranks split them with no data-path exchange; only
scalar counters and timings are reduced on the host."""
from __future__ import annotations

from typing import Tuple

import numpy as np


def frame_offset(rank: int, batch: int, frames_per_batch: int, batches: int) -> int:
    """First global frame index of `batch` on `rank` when every rank decodes
    its own `batches` batches of `frames_per_batch` frames (weak scaling)."""
    if rank < 0 or batch < 0 or batch >= batches or frames_per_batch < 0:
        raise ValueError("bad shard arguments")
    return (rank * batches + batch) * frames_per_batch


def shard_range(total: int, rank: int, world: int) -> Tuple[int, int]:
    """(start, count) of rank's contiguous share of `total` frames (strong
    scaling): the first total % world ranks take one extra frame."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def mixed_shard(code_of_frame_all, rank: int, world: int):
    """Rank's frames of a mixed batch under weak scaling: the global
    assignment holds world * F frames (F per rank); rank r decodes frames
    r F .. (r + 1) F - 1, keeping their codes and order.  Returns (first
    global frame, the rank's code-of-frame array)."""
    cof = np.asarray(code_of_frame_all)
    if world < 1 or not 0 <= rank < world or cof.size % world:
        raise ValueError("bad shard arguments")
    per = cof.size // world
    return rank * per, np.ascontiguousarray(cof[rank * per:(rank + 1) * per], dtype=np.int32)


def reduce_counters(counters, op: str = "sum"):
    """All-reduce an int64 counter vector over the default process group
    (a no-op without one); returns a numpy array."""
    import torch
    import torch.distributed as dist
    arr = np.asarray(counters, dtype=np.int64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return arr.copy()
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.from_numpy(arr.copy()).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return t.cpu().numpy()
