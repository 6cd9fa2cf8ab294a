"""Experiment runners built on the hot path (paper Sec. III-IV).

* throughput_vs_n: wall time of a fixed propagation time against the ensemble
  size N (the measurement of Fig. 1; the paper's curve steps at multiples of
  the number of realisations its GPU ran at once).
* web_density: the Arnold-web picture of Figs. 2-3 - an ensemble uniform over
  (a patch of) the momentum sphere, V over one window, F as a histogram of the
  direction of V, optionally only trajectories that stayed in the patch.
* diffusion_from_w: Fig. 4 - a Gaussian cloud at the triple resonance
  W = (sqrt E, sqrt E, 0), windows of dt, F time-averaged between snapshots,
  with checkpoint/resume for long horizons.
"""
from __future__ import annotations

import math
import os

import numpy as np

from .api import ArnoldEnsemble
from .params import paper_h

T = 2.0 * math.pi


def throughput_vs_n(ns, steps: int = 200, precision: str = "fp64", E: float = 400.0, tangent: bool = True,
                    device: int = 0) -> list[dict]:
    """Time `steps` composite steps for each ensemble size in ns (sphere ICs at E)."""
    import torch
    out = []
    for n in ns:
        e = ArnoldEnsemble(int(n), precision=precision, tangent=tangent, device=device)
        e.init_sphere(E, seed=1)
        e.iterate(min(steps, 10))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        e.iterate(steps)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        out.append({"n": int(n), "ms": ms, "ms_per_step": ms / steps, "map_steps_per_s": n * steps / (ms * 1e-3)})
        e.close()
    return out


def web_density(n: int, E: float, window_T: float = 50.0, n_cos: int = 256, n_phi: int = 512,
                patch=(-1.0, 1.0, 0.0, 2 * math.pi), track: bool = False, precision: str = "fp32c",
                seed: int = 0, h: float | None = None, device: int = 0) -> dict:
    """Figs. 2-3: ICs uniform over the patch of S and over the torus, propagated
    for t_p = dt = window_T periods; returns the counts of V's direction on the
    patch (and the fraction of trajectories kept by the area filter)."""
    h = paper_h() if h is None else h
    steps = int(round(window_T * T / h))
    e = ArnoldEnsemble(n, precision=precision, tangent=False, h=h, window=steps, device=device)
    e.init_sphere(E, seed=seed, cos_range=patch[:2], phi_range=patch[2:])
    if track:
        e.track_patch(*patch)
    e.iterate(steps)
    counts = e.velocity_histogram(n_cos, n_phi, patch=patch, filtered=track)
    kept = 1.0 - float(np.mean(e.indicator("left"))) if track else 1.0
    e.sync()
    return {"counts": counts, "steps": steps, "kept_fraction": kept, "n": n, "E": E}


def diffusion_from_w(n: int = 32000, E: float = 15.0, sigma: float = 0.01, window_T: float = 50.0,
                     snapshots_T=(1e2, 1e3, 1e4), n_cos: int = 128, n_phi: int = 256, precision: str = "df64f",
                     seed: int = 0, ckpt_path: str | None = None, device: int = 0, h: float | None = None) -> dict:
    """Fig. 4: the cloud starts at W = (sqrt E, sqrt E, 0) with Gaussian (p_x, p_y)
    of width sigma and p_z from the energy; angles whose energy condition has no
    real p_z are redrawn (the cloud sits where |P|^2 = 2E, so the potential must
    be <= 0 there).  F of V over windows of window_T is accumulated between
    consecutive snapshot times (time-averaged F).  With ckpt_path the state, the
    window count and the accumulated F are saved together after every window
    (one file, replaced atomically) and a rerun resumes from it.  The default
    precision is the long-horizon double-float mode: the run reaches 1e9 steps,
    where FP32C's energy error walks to ~1e-2."""
    import torch
    h = paper_h() if h is None else h
    W = math.sqrt(E)
    w_steps = int(round(window_T * T / h))
    e = init_gaussian_valid(n, E, (W, W), sigma, seed, precision=precision, window=w_steps, h=h, device=device)
    done_windows = 0
    maps = []
    # F accumulates on the device between snapshots (no host round trip per window)
    acc = torch.zeros((n_cos, n_phi), dtype=torch.int64, device=f"cuda:{device}")
    bounds = [int(round(s * T / h / w_steps)) for s in snapshots_T]
    if ckpt_path and os.path.exists(ckpt_path):
        done_windows, acc_np = _load_fig4_ckpt(ckpt_path, e, bounds, (n_cos, n_phi))
        acc.copy_(torch.from_numpy(acc_np))
    k = 0
    while k < len(bounds) and bounds[k] <= done_windows:
        k += 1
    while k < len(bounds):
        e.iterate(w_steps)
        done_windows += 1
        e.velocity_histogram(n_cos, n_phi, out=acc, accumulate=True)
        if done_windows == bounds[k]:
            maps.append({"t_T": snapshots_T[k], "counts": acc.cpu().numpy().astype(np.uint64)})
            acc.zero_()
            k += 1
        if ckpt_path:
            _save_fig4_ckpt(ckpt_path, e, done_windows, acc.cpu().numpy())
    e.sync()
    return {"maps": maps, "windows": done_windows, "n": n, "E": E, "window_steps": w_steps,
            "dE_max": float(e.indicator("dE_max").max())}


def _save_fig4_ckpt(path: str, e: ArnoldEnsemble, done_windows: int, acc: np.ndarray) -> None:
    """Ensemble checkpoint, window count and accumulated F in one file, written
    to a private temporary and renamed over `path`: a crash leaves either the
    previous checkpoint or the new one, never a mix."""
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as f:
        np.savez(f, state=np.frombuffer(e.checkpoint(), dtype=np.uint8), done_windows=np.int64(done_windows),
                 acc=acc.astype(np.int64))
    os.replace(tmp, path)


def _load_fig4_ckpt(path: str, e: ArnoldEnsemble, bounds, shape):
    """Restore a Fig. 4 checkpoint into `e`; returns (done_windows, acc).  The
    accumulated F must hold exactly the windows since the last snapshot
    boundary, and have the run's F shape; anything else is an error."""
    with np.load(path) as z:
        if set(z.files) != {"state", "done_windows", "acc"}:
            raise ValueError(f"{path}: not a Fig. 4 checkpoint")
        done = int(z["done_windows"])
        acc = z["acc"].astype(np.int64)
        state = z["state"].tobytes()
    if acc.shape != tuple(shape):
        raise ValueError(f"{path}: F shape {acc.shape} != {tuple(shape)}")
    last = max([b for b in bounds if b <= done], default=0)
    n_acc = int(acc.sum())
    if done > last and n_acc == 0:
        raise ValueError(f"{path}: F holds no window since window {last}, but {done} windows are done")
    if done == last and n_acc != 0:
        raise ValueError(f"{path}: F is not empty at a snapshot boundary")
    e.restore(state)
    return done, acc


def init_gaussian_valid(n: int, E: float, center, sigma: float, seed: int, **kw) -> ArnoldEnsemble:
    """Gaussian cloud with p_z from the energy (Fig. 4), drawn on the device:
    draws whose energy condition has no real solution are skipped, the first n
    that have one are kept in draw order (arnold_init_gaussian)."""
    e = ArnoldEnsemble(n, tangent=False, **kw)
    e.init_gaussian(E, center, sigma, seed)
    return e


SWEEP_NS = [1, 32, 148, 1024, 4736, 9472, 9473, 18944, 37888, 75776, 151552, 151553, 303104, 606208, 1048576,
            4194304, 10000000]


def timed_web_experiment(n: int, E: float = 400.0, window_T: float = 50.0, precision: str = "fp64",
                         n_cos: int = 256, n_phi: int = 512, seed: int = 0, device: int = 0) -> dict:
    """One web experiment of Sec. IV at a given scale (the paper's: N ~ 1e8, t_p =
    dt = 50 T = 5000 steps, FP64): sphere ICs, propagation, F.  Returns the
    host set-up time, the propagation time (CUDA events on the ensemble's
    stream) and the histogram time."""
    import time

    import torch
    h = paper_h()
    steps = int(round(window_T * T / h))
    st = torch.cuda.current_stream(device)
    t0 = time.perf_counter()
    e = ArnoldEnsemble(n, precision=precision, tangent=False, h=h, window=steps, device=device,
                       stream=st.cuda_stream)
    e.init_sphere(E, seed=seed)
    e.sync()
    t_init = time.perf_counter() - t0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    e.iterate(steps)
    b.record(st)
    b.synchronize()
    e.sync()
    t_prop = a.elapsed_time(b) * 1e-3
    t1 = time.perf_counter()
    counts = e.velocity_histogram(n_cos, n_phi)
    t_hist = time.perf_counter() - t1
    e.close()
    return {"n": n, "E": E, "steps": steps, "precision": precision, "init_s": t_init, "propagate_s": t_prop,
            "map_steps_per_s": n * steps / t_prop, "histogram_s": t_hist, "counted": int(counts.sum())}


def scan_agreement(E: float = 400.0, steps: int = 1_000_000, G: int = 2048,
                   precisions=("fp64", "fp32c", "df64", "df64f"),
                   seed: int = 0, device: int = 0) -> list[dict]:
    """The Arnold-web scan of Sec. IV on a G x G grid of initial actions at
    energy E, run to `steps` steps in every precision mode from the same initial
    conditions; per mode the time, chaotic fraction and, against the first mode,
    class agreement and the L1 distance of the log10 chi histograms.

    "fp64ulp" is FP64 from the grid's angles moved up by one ulp (p_z again
    from the energy; z moves by exactly one ulp, x and y through the rotated
    angles u = x + y, v = x - y at their rounding): against "fp64" it gives the
    agreement any two runs that round differently can reach on this field."""
    return list(iter_scan_agreement(E, steps, G, precisions, seed, device))


def iter_scan_agreement(E: float = 400.0, steps: int = 1_000_000, G: int = 2048,
                        precisions=("fp64", "fp32c", "df64", "df64f"), seed: int = 0, device: int = 0):
    """scan_agreement, one mode's record at a time as each run finishes."""
    import torch
    st = torch.cuda.current_stream(device)
    ref = None
    for prec in precisions:
        e = ArnoldEnsemble(G * G, precision="fp64" if prec == "fp64ulp" else prec, device=device,
                           stream=st.cuda_stream)
        if prec == "fp64ulp":
            raw = torch.empty((6, G * G), dtype=torch.float64, device=f"cuda:{device}")
            e.init_grid(G, E, seed=seed, raw_out=raw)
            st.synchronize()
            X = torch.nextafter(raw[:3], torch.full_like(raw[:3], math.inf)).contiguous()
            e.set_state_shell(X, raw[3:].contiguous(), 2, E)
            st.synchronize()
            del raw, X
        else:
            e.init_grid(G, E, seed=seed)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        e.iterate(steps)
        b.record(st)
        b.synchronize()
        e.sync()
        chi, cls = e.indicator("chi"), e.indicator("class")
        dev = e.indicator("vdev")
        rank = lambda v: np.argsort(np.argsort(v)).astype(np.float64)  # noqa: E731
        r = {"precision": prec, "E": E, "G": G, "steps": steps, "seconds": a.elapsed_time(b) * 1e-3,
             "map_steps_per_s": G * G * steps / (a.elapsed_time(b) * 1e-3), "chaotic_fraction": float(cls.mean()),
             "dE_max": float(e.indicator("dE_max").max()),
             # Sec. IV's reading of V beside chi: |V - P(0)| of chaotic vs regular cells, and its rank
             # correlation with chi (reported)
             "vdev_median_chaotic": float(np.median(dev[cls == 1])) if cls.any() else None,
             "vdev_median_regular": float(np.median(dev[cls == 0])) if (cls == 0).any() else None,
             "vdev_chi_rank_correlation": float(np.corrcoef(rank(dev), rank(chi))[0, 1])}
        if ref is None:
            ref = (chi, cls)
        else:
            h = lambda c: np.histogram(np.log10(np.clip(c, 1e-300, None)), bins=200, range=(-8, 1))[0] / c.size
            r["class_agreement"] = float(np.mean(cls == ref[1]))
            r["hist_l1"] = float(np.abs(h(chi) - h(ref[0])).sum())
        e.close()
        yield r


def timed_diffusion_rate(n: int = 32000, E: float = 15.0, steps: int = 50000, precision: str = "fp64",
                         sigma: float = 0.01, seed: int = 0, device: int = 0) -> dict:
    """Rate of the long diffusion run of Fig. 4 (the cloud at W, no tangent) over
    `steps` steps, and the projected time of the paper's 1e9 steps at that rate."""
    import torch
    st = torch.cuda.current_stream(device)
    e = init_gaussian_valid(n, E, (math.sqrt(E), math.sqrt(E)), sigma, seed, precision=precision,
                            window=int(round(50 * T / paper_h())), device=device, stream=st.cuda_stream)
    e.iterate(100)                       # warm-up
    e.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    e.iterate(steps)
    b.record(st)
    b.synchronize()
    e.sync()
    sec = a.elapsed_time(b) * 1e-3
    rate = n * steps / sec
    e.close()
    return {"n": n, "E": E, "steps": steps, "precision": precision, "seconds": sec, "map_steps_per_s": rate,
            "projected_1e9_steps_h": n * 1e9 / rate / 3600.0}


def main(argv=None):
    """python -m paper_1107_4107_b300.experiments sweep [PREC,PREC,...]
           -> JSON lines of throughput_vs_n (default: every precision mode)
       python -m paper_1107_4107_b300.experiments web N PRECISION [E]
           -> one timed web experiment (sphere, 5000 steps, F) as a JSON line
       python -m paper_1107_4107_b300.experiments diffusion PRECISION
           -> the Fig. 4 diffusion run's rate (32,000 trajectories, E = 15)
       python -m paper_1107_4107_b300.experiments fig4 PRECISION T_END [OUT.npz]
           -> the Fig. 4 run itself to T_END periods: F time-averaged between
              the snapshot times 1e2, 1e3, ... T (saved to OUT.npz), wall time
       python -m paper_1107_4107_b300.experiments scan E STEPS [G [PREC,PREC,...]]
           -> the G x G scan in FP64, FP32C, DF64 and DF64F (or the listed modes) with agreement vs FP64"""
    import json
    import sys
    args = sys.argv[1:] if argv is None else argv
    if args and args[0] == "scan" and len(args) >= 3:
        precs = tuple(args[4].split(",")) if len(args) > 4 else ("fp64", "fp32c", "df64", "df64f")
        for r in iter_scan_agreement(E=float(args[1]), steps=int(float(args[2])),
                                     G=int(args[3]) if len(args) > 3 else 2048, precisions=precs):
            print(json.dumps(r), flush=True)
        return
    if args and args[0] == "fig4" and len(args) >= 3:
        import time
        t_end = float(args[2])
        snaps = tuple(t for t in (1e2, 1e3, 1e4, 1e5, 1e6, 1e7) if t <= t_end)
        t0 = time.perf_counter()
        r = diffusion_from_w(precision=args[1], snapshots_T=snaps)
        wall = time.perf_counter() - t0
        if len(args) > 3:
            np.savez_compressed(args[3], **{f"F_{int(m['t_T'])}T": m["counts"] for m in r["maps"]})
        print(json.dumps({"precision": args[1], "n": r["n"], "E": r["E"], "t_end_T": t_end,
                          "steps": r["windows"] * r["window_steps"], "wall_s": wall,
                          "map_steps_per_s": r["n"] * r["windows"] * r["window_steps"] / wall,
                          "dE_max": r["dE_max"],
                          "snapshots": [{"t_T": m["t_T"], "occupied_cells": int(np.count_nonzero(m["counts"])),
                                         "counts": int(m["counts"].sum())} for m in r["maps"]]}), flush=True)
        return
    if args and args[0] == "diffusion" and len(args) >= 2:
        print(json.dumps(timed_diffusion_rate(precision=args[1])), flush=True)
        return
    if args and args[0] == "web" and len(args) >= 3:
        r = timed_web_experiment(int(float(args[1])), E=float(args[3]) if len(args) > 3 else 400.0,
                                 precision=args[2])
        print(json.dumps(r), flush=True)
        return
    if not args or args[0] != "sweep":
        raise SystemExit("usage: python -m paper_1107_4107_b300.experiments sweep [PRECISIONS] | web N PRECISION [E] | "
                         "diffusion PRECISION | fig4 PRECISION T_END [OUT] | scan E STEPS [G [PRECISIONS]]")
    steps = {"fp64": (200, 50), "fp32c": (1000, 400), "df64": (400, 100), "df64f": (600, 150)}   # (N <= 606,208, larger N)
    for prec in (args[1].split(",") if len(args) > 1 else ("fp64", "fp32c", "df64", "df64f")):
        small = [n for n in SWEEP_NS if n <= 606208]
        big = [n for n in SWEEP_NS if n > 606208]
        rows = throughput_vs_n(small, steps=steps[prec][0], precision=prec)
        rows += throughput_vs_n(big, steps=steps[prec][1], precision=prec)
        for r in rows:
            r["precision"] = prec
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
