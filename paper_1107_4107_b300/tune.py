"""Autotuner of the batched persistent launch.

Times each candidate (block size, trajectories per thread, renormalisation
interval) on a scaled-down copy of the batch (G / 4, n_steps / 200) with CUDA
events and keeps the fastest.  Results are cached per (GPU name, precision,
scheme, tangent) in tune_cache.json next to this file.  The renormalisation
interval only changes rounding of the FTLE (chi is independent of R) and the
sampling interval of the energy error; candidates stay below R h lambda ~ 50,
so the FP32 tangent cannot overflow between renormalisations.  The
double-float modes run one trajectory per thread.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tune_cache.json")
CANDIDATES = [{"block_size": b, "traj_per_thread": t, "renorm_every": r, "epoch_ms": 200}
              for b in (128, 256) for t in (1, 2) for r in (50, 100, 200)]


def candidates_for(precision: str):
    return [c for c in CANDIDATES if precision == "fp32c" or c["traj_per_thread"] == 1]


def _key(precision: str, scheme: str, tangent: bool, device: int) -> str:
    import torch
    return f"{torch.cuda.get_device_name(device)}|{precision}|{scheme}|{int(tangent)}"


def scaled(sets, g_div: int = 4, step_div: int = 200):
    return [dict(q, G=max(8, int(q["G"]) // g_div), n_steps=max(16, int(q["n_steps"]) // step_div)) for q in sets]


def tune_batch(sets, scheme: str = "yoshida6a", tangent: bool = True, use_cache: bool = True,
               candidates=None, verbose: bool = False, device: int | None = None, precision: str = "fp32c") -> dict:
    """Best tuning for `sets` in `precision` on `device` (default: torch's current device)."""
    import torch
    from .api import ArnoldBatch
    if device is None:
        device = torch.cuda.current_device()
    key = _key(precision, scheme, tangent, device)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                cache = json.load(f)
        except ValueError:
            cache = {}
        if key in cache:
            return cache[key]["tuning"]
    sample = scaled(sets)
    results = []
    stream = torch.cuda.current_stream(device)
    for cand in candidates or candidates_for(precision):
        b = ArnoldBatch(sample, scheme=scheme, tangent=tangent, tuning=cand, device=device,
                        stream=stream.cuda_stream, precision=precision)
        b.init()
        b.run()          # captures the graph, warms up
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run()
        e1.record(stream)
        b.sync()
        ms = e0.elapsed_time(e1)
        rate = b.info()["map_steps_per_run"] / (ms * 1e-3)
        results.append((rate, cand))
        if verbose:
            print(f"tune {cand}: {rate:.3e} map-steps/s")
        b.close()
    best = max(results, key=lambda r: r[0])
    cache[key] = {"tuning": best[1], "rate_sample": best[0],
                  "all": [{"tuning": c, "rate": r} for r, c in results]}
    if use_cache:
        # several processes (one per GPU) may tune at once: write a private file
        # and rename it over the cache, so a reader never sees a partial file
        tmp = f"{CACHE}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, CACHE)
    return best[1]
