"""A small, fixed case of the hot path for profilers (ncu) and quick timing.

    python -m paper_1107_4107_b300.profile_case --precision fp64 --n 1048576 --steps 20 --launches 3
    python -m paper_1107_4107_b300.profile_case --batch 0.01 --launches 2 [--batch-precision df64f]

Grid-slice ICs at E = 400 (the scan's initial conditions on a sqrt(n)-wide
band of the 2048-wide grid), then `launches` calls of iterate(steps), each one
kernel launch; prints the mean launch time from CUDA events.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32c", "df64", "df64f"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--no-tangent", action="store_true")
    ap.add_argument("--adjoint", type=int, default=0, metavar="C",
                    help="instead: the FP64/FP32C adjoint of the variance loss over --steps steps of --n box "
                         "trajectories with checkpoints every C steps (one k_adjoint launch per segment)")
    ap.add_argument("--batch", type=float, default=0.0, metavar="SCALE",
                    help="instead: the 64-set batch with steps scaled by SCALE and a fixed tuning "
                         "(block 128, 1 trajectory per thread, R 200, 200 ms epochs): --launches graph runs")
    ap.add_argument("--batch-precision", default="fp32c", choices=["fp32c", "df64f", "df64"])
    a = ap.parse_args()
    import torch
    from .api import ArnoldEnsemble
    if a.batch:
        from . import params
        from .api import ArnoldBatch
        b = ArnoldBatch(params.batch_sets(step_scale=a.batch),
                        tuning={"block_size": 128, "traj_per_thread": 1, "renorm_every": 200, "epoch_ms": 200},
                        stream=torch.cuda.current_stream().cuda_stream, precision=a.batch_precision)
        times = []
        for _ in range(a.launches):
            b.init()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.run()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        b.sync()
        info = b.info()
        print(json.dumps({"batch": a.batch, "precision": a.batch_precision, "ms": times, "epochs": info["epochs"], "items": info["items"],
                          "map_steps_per_s": info["map_steps_per_run"] / (min(times) * 1e-3)}))
        return
    if a.adjoint:
        from . import inputs
        X, P = inputs.box(a.n, seed=0)
        e = ArnoldEnsemble(a.n, precision=a.precision, tangent=False, stream=torch.cuda.current_stream().cuda_stream)
        e.set_state(X, P)
        e.forward_ckpt(a.steps, a.adjoint)
        PN = torch.empty((3, a.n), device="cuda", dtype=torch.float64)
        e.indicator("P", out=PN)
        up = ((2.0 / 3.0) * (PN - PN.mean(dim=1, keepdim=True)) / a.n).contiguous()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        g = e.grad(dL_dp=up)
        t1.record()
        t1.synchronize()
        print(json.dumps({"adjoint": a.precision, "n": a.n, "steps": a.steps, "ckpt_every": a.adjoint,
                          "reverse_ms": t0.elapsed_time(t1), "dL_dh": float(g[2])}))
        return
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
