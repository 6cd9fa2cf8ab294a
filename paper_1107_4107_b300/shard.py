"""Multi-rank host logic: how a scan is split over ranks and how their
ensemble statistics are merged.

The path partitions into independent trajectories.  A sharded scan gives rank
r a contiguous band of grid rows (arnold_init_grid's row0), so every rank
draws exactly the initial conditions the single-GPU scan would; the only
exchange is the final sum of statistics, merged on the host in FP64 in rank
order (Chan et al. for the moments), so the result does not depend on timing.
"""
from __future__ import annotations

import numpy as np


def row_band(G: int, rank: int, world: int) -> tuple[int, int]:
    """(row0, rows) of rank's contiguous band of a G-row grid (sizes differ by <= 1)."""
    if not (0 <= rank < world) or G < world:
        raise ValueError("need 0 <= rank < world <= G")
    base, extra = divmod(G, world)
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def merge_stats(parts: list[dict]) -> dict:
    """Merge per-shard statistics dicts (hist, under, over, chaotic, n, dE_max,
    p_mean, p_var), in list order."""
    out = {"hist": np.zeros_like(np.asarray(parts[0]["hist"])), "under": 0, "over": 0, "chaotic": 0, "n": 0,
           "dE_max": 0.0, "p_mean": np.zeros(3), "p_var": np.zeros(3)}
    m2 = np.zeros(3)
    for p in parts:
        nb = int(p["n"])
        if nb == 0:
            continue
        na = out["n"]
        mb = np.asarray(p["p_mean"], dtype=np.float64)
        m2b = np.asarray(p["p_var"], dtype=np.float64) * nb
        d = mb - out["p_mean"]
        tot = na + nb
        out["p_mean"] = out["p_mean"] + d * (nb / tot)
        m2 = m2 + m2b + d * d * (na * nb / tot)
        out["n"] = tot
        out["hist"] = out["hist"] + np.asarray(p["hist"])
        for k in ("under", "over", "chaotic"):
            out[k] += int(p[k])
        out["dE_max"] = max(out["dE_max"], float(p["dE_max"]))
    out["p_var"] = m2 / out["n"] if out["n"] else m2
    return out


def gather_stats(stats: dict, group=None) -> dict | None:
    """All-gather every rank's statistics over torch.distributed and merge them in
    rank order on every rank (host objects: works with gloo and nccl)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, {k: (np.asarray(v).tolist() if isinstance(v, np.ndarray) else v)
                                   for k, v in stats.items()}, group=group)
    return merge_stats(parts)
