"""Replica sharding of the detection path over several GPUs (one process per GPU).

Frames are independent units of work, so the path shards without any collective on the data path: the
frame sequence is partitioned round-robin over the ranks, every rank detects its own frames with its own
library handle on its own GPU, and the host gathers the 192-byte per-frame result records (``ld_lanes``)
on rank 0.  Timing takes the slowest rank.  The only collectives are these host-side exchanges, so the
same code runs over ``gloo`` (CPU) or ``nccl``.
"""
from __future__ import annotations

import numpy as np

from .ld import LANES_DTYPE


def frames_of_rank(n_frames: int, rank: int, world: int) -> list[int]:
    """Round-robin partition: rank r takes frames r, r + world, r + 2 world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    return list(range(rank, n_frames, world))


def _dist():
    import torch.distributed as dist

    return dist if dist.is_available() and dist.is_initialized() else None


def gather_lanes(local: np.ndarray, frames: list[int], n_frames: int) -> np.ndarray | None:
    """Gather every rank's result records on rank 0, in frame order.

    local: LANES_DTYPE records of this rank, one per entry of ``frames``.  Returns the n_frames records on
    rank 0 and None elsewhere (with no process group, the local records, which must then cover every frame).
    """
    local = np.ascontiguousarray(local, dtype=LANES_DTYPE)
    if len(local) != len(frames):
        raise ValueError("one record per frame expected")
    dist = _dist()
    parts = [(list(frames), local.tobytes())]
    if dist is not None and dist.get_world_size() > 1:
        gathered = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
        dist.gather_object(parts[0], gathered, dst=0)
        if dist.get_rank() != 0:
            return None
        parts = gathered
    out = np.zeros(n_frames, LANES_DTYPE)
    seen = np.zeros(n_frames, bool)
    for idx, raw in parts:
        rec = np.frombuffer(raw, LANES_DTYPE)
        if len(rec) != len(idx):
            raise ValueError("record count does not match the frame list")
        for k, fidx in enumerate(idx):
            if seen[fidx]:
                raise ValueError(f"frame {fidx} reported by two ranks")
            seen[fidx] = True
            out[fidx] = rec[k]
    if not seen.all():
        raise ValueError(f"frames without a result: {np.flatnonzero(~seen)[:8].tolist()}")
    return out


def max_over_ranks(x: float) -> float:
    """The largest value of x over the ranks (the slowest rank's time); x itself without a process group."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
