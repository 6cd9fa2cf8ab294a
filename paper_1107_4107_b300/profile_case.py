"""A small, fixed case of the hot path for profilers (ncu) and quick timing.

    python -m paper_1107_4107_b300.profile_case --precision fp64 --n 1048576 --steps 20 --launches 3

Grid-slice ICs at E = 400 (the scan's initial conditions on a sqrt(n)-wide
band of the 2048-wide grid), then `launches` calls of iterate(steps), each one
kernel launch; prints the mean launch time from CUDA events.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32c", "df64"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--no-tangent", action="store_true")
    a = ap.parse_args()
    import torch
    from .api import ArnoldEnsemble
    G = 2048
    if a.n % G:
        raise SystemExit("--n must be a multiple of 2048")
    ens = ArnoldEnsemble(a.n, precision=a.precision, tangent=not a.no_tangent, launch_steps=a.steps,
                         stream=torch.cuda.current_stream().cuda_stream)
    ens.init_grid(G, 400.0, row0=0)
    st = torch.cuda.current_stream()
    times = []
    for _ in range(a.launches):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ens.iterate(a.steps)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ens.sync()
    print(json.dumps({"precision": a.precision, "n": a.n, "steps": a.steps, "ms": times,
                      "map_steps_per_s": a.n * a.steps / (min(times) * 1e-3)}))


if __name__ == "__main__":
    main()
