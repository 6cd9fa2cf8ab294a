"""Multi-rank host logic: how a scan is split over ranks and how their
ensemble statistics and adjoint partials are merged.

The path partitions into independent trajectories.  A sharded scan gives rank
r a contiguous band of grid rows (arnold_init_grid's row0), so every rank
draws exactly the initial conditions the single-GPU scan would; the only
exchange is the final sum of statistics, merged on the host in FP64 in rank
order (Chan et al. for the moments), so the result does not depend on timing.

The adjoint of the variance loss L = (1/3) sum_alpha Var_i P_alpha(N) couples
all trajectories through the ensemble mean, so a sharded gradient has two
exchanges: the loss partials (count, mean, M2 per component) before the
reverse sweep, which give every rank the global mean and its upstream
dL/dP_i = (2/3)(P_i - mean)/N, and the (dL/dh, dL/deps) partials after it,
summed exactly (math.fsum) in rank order.  Per-trajectory gradients stay on
their rank.
"""
from __future__ import annotations

import math

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


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def loss_partials(P) -> dict:
    """This shard's share of the variance loss: count, per-component mean and
    M2 = sum (P - mean)^2 of its final momenta P [3][n_local]."""
    P = _host(P)
    n = int(P.shape[1])
    mean = P.mean(axis=1) if n else np.zeros(3)
    m2 = ((P - mean[:, None]) ** 2).sum(axis=1) if n else np.zeros(3)
    return {"n": n, "mean": mean.tolist(), "m2": m2.tolist()}


def combine_loss(parts: list[dict]) -> dict:
    """Merge loss partials in list (rank) order (Chan et al.): global count N,
    mean, population variance and L = (1/3) sum_alpha Var_alpha."""
    n, mean, m2 = 0, np.zeros(3), np.zeros(3)
    for p in parts:
        nb = int(p["n"])
        if nb == 0:
            continue
        mb, m2b = np.asarray(p["mean"]), np.asarray(p["m2"])
        d = mb - mean
        tot = n + nb
        mean = mean + d * (nb / tot)
        m2 = m2 + m2b + d * d * (n * nb / tot)
        n = tot
    var = m2 / n if n else m2
    return {"n": n, "mean": mean, "var": var, "loss": float(var.sum() / 3.0)}


def loss_upstream(P, combined: dict):
    """dL/dP_i = (2/3)(P_i - mean)/N for this shard's trajectories (same type and
    device as P: numpy, or a torch tensor)."""
    scale = 2.0 / (3.0 * combined["n"])
    if hasattr(P, "detach"):
        import torch
        mean = torch.as_tensor(combined["mean"], dtype=P.dtype, device=P.device)[:, None]
        return ((P - mean) * scale).contiguous()
    return (_host(P) - np.asarray(combined["mean"])[:, None]) * scale


def combine_param_grads(parts) -> tuple[float, float]:
    """Sum the shards' (dL/dh, dL/deps) partials exactly (math.fsum)."""
    return math.fsum(float(p[0]) for p in parts), math.fsum(float(p[1]) for p in parts)


def variance_loss_grad(P, local_backward, exchange):
    """Sharded gradient of the variance loss.  P: this shard's final momenta;
    local_backward(upstream) -> (g_x0, g_p0, g_h, g_eps) of this shard's
    trajectories (e.g. ArnoldEnsemble.grad after forward_ckpt);
    exchange(obj) -> every shard's obj in rank order.  Returns (L, g_x0, g_p0,
    g_h, g_eps) with g_h, g_eps summed over all shards."""
    comb = combine_loss(exchange(loss_partials(P)))
    gx, gp, gh, ge = local_backward(loss_upstream(P, comb))
    gh_t, ge_t = combine_param_grads(exchange((float(gh), float(ge))))
    return comb["loss"], gx, gp, gh_t, ge_t


def dist_exchange(group=None):
    """exchange() over torch.distributed: all-gather of host objects in rank order
    (gloo or nccl)."""
    import torch.distributed as dist

    def ex(obj):
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, obj, group=group)
        return parts
    return ex
