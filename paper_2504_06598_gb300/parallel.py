"""Sharding the stochastic renderer's rays over ranks (one process per GPU).

Rays are independent (Sec. 3.4), so the work shards by view with the scene
replicated on every rank and no collective on the data path; the only
communication is the timing reduction of a benchmark. Ray ids stay globally
unique, so every rank's draws differ and the results do not depend on the
number of ranks.
"""

from __future__ import annotations

import os
from dataclasses import replace

import torch


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_views(cams, rank: int, world: int):
    """Views of this rank (round robin), keeping their global ray ids.

    ``cams`` must already have disjoint ray-id ranges (as produced by
    ``scenes.orbit_cameras`` / ``scenes.wavefront_views``)."""
    return [c for i, c in enumerate(cams) if i % world == rank]


def rank_view(cam, rank: int):
    """The benchmark's weak scaling: every rank renders the same camera with
    its own block of ray ids (rank * width * height onwards)."""
    return replace(cam, ray_id_offset=int(cam.ray_id_offset) + rank * cam.width * cam.height)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity when
    torch.distributed is not initialised)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]
