"""Write the oracle's long-horizon FTLE values on sampled cells of the 2048 x 2048
scan (tests/golden/oracle_scan_2048_1e6.json).

    python tests/golden/make_oracle_scan_1e6.py [--threads T] [--cells K]
    python tests/golden/make_oracle_scan_1e6.py --energy 15     # add one energy to the record
    python tests/golden/make_oracle_scan_1e6.py --ulp 40        # the one-ulp run (below)

The FP64 Arnold-web scan (Sec. IV: the web drawn over a 2-D slice of initial
actions; Sec. III: sixth-order map at h = 0.01 T) runs 1e6 composite steps on
a 2048 x 2048 grid, far beyond what the CPU oracle can do in full.  This script
runs the oracle -- and nothing else -- over a seeded subset of K = 4096 grid
cells at E = 400 (eps_eff = 0.005, the weak value), E = 40 (10x that) and
E = 15 (eps_eff = 2/15, the paper's moderate value), from
the grid's own initial conditions (seeded angles, (p_x, p_y) at the cell
centre, p_z from the energy), with the tangent renormalised every 100 steps,
and records chi_t at 1e4, 1e5 and 1e6 steps (and the log-sum at 1e6).  The
GPU tests compare their own runs of the same cells with these values
(classification agreement and histogram L1 of log10 chi).

With --energy E (repeatable) it runs only those energies and merges them into
the existing record, whose grid, cells and marks must be the same.

With --ulp E it instead runs the oracle at energy E from the same cells with
every initial angle moved up by one ulp, and writes its chi at the same marks
to tests/golden/oracle_scan_2048_1e6_ulp.json: where some cells are chaotic,
their finite-time exponents decorrelate under any rounding difference, so the
oracle against itself gives the agreement level the indicator allows on this
sample.

Inputs come from the seeded generator module only; every number written here
comes from oracle/.  ~4.1e9 map steps per energy: about 20 minutes per energy
on 8 host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1107_4107_b300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_scan_2048_1e6.json")
OUT_ULP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_scan_2048_1e6_ulp.json")
G = 2048
ENERGIES = (400.0, 40.0, 15.0)
EPS = 1.0
H = 0.02 * math.pi
R = 100
SEED = 0            # initial angles of the grid
SAMPLE_SEED = 2048  # which cells
MARKS = (10_000, 100_000, 1_000_000)


def cells(k: int) -> np.ndarray:
    return inputs.sample_cells(G * G, k, seed=SAMPLE_SEED)


def initial_state(E: float, idx: np.ndarray, ulp: bool = False):
    """Grid-slice ICs of the sampled cells (angles and (p_x, p_y) from the seeded
    generator, p_z from the fixed-energy condition computed by the oracle);
    ulp: every angle moved up by one ulp first."""
    X, Pxy = inputs.grid_slice(G, E, EPS, seed=SEED)
    X = X[:, idx].copy()
    if ulp:
        X = np.nextafter(X, np.inf)
    P = np.zeros((3, len(idx)))
    P[:2] = Pxy[:, idx]
    return X, oracle.pz_from_energy(E, EPS, X, P)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--cells", type=int, default=4096)
    ap.add_argument("--out", default=None)
    ap.add_argument("--energy", type=float, action="append", default=None, metavar="E",
                    help="run only energy E and merge it into the existing record (repeatable)")
    ap.add_argument("--ulp", type=float, action="append", default=None, metavar="E",
                    help="run the one-ulp-perturbed oracle at energy E instead (repeatable)")
    args = ap.parse_args()
    idx = cells(args.cells)
    if args.ulp:
        return run_ulp(args, idx)
    rec = {"what": "oracle chi_t (FTLE, tangent renormalised every R steps) on sampled cells of the 2048x2048 "
                   "grid slice; written by tests/golden/make_oracle_scan_1e6.py from oracle/ only",
           "grid": G, "eps": EPS, "h": H, "renorm_every": R, "scheme": "yoshida6a", "seed": SEED,
           "sample_seed": SAMPLE_SEED, "cells": len(idx),
           "cells_sha256": hashlib.sha256(idx.astype("<i8").tobytes()).hexdigest(),
           "marks": list(MARKS), "energies": {}}
    out = args.out or OUT
    if args.energy:
        rec = _merge_base(rec, out)
    for E in args.energy or ENERGIES:
        X, P = initial_state(E, idx)
        st = oracle.State(X, P, oracle.Params(eps=EPS, h=H, renorm_every=R))
        row = {"chi": {}}
        t0 = time.perf_counter()
        for m in MARKS:
            while st.steps < m:
                st.advance(min(100_000, m - st.steps), threads=args.threads)
            row["chi"][str(m)] = [float(f"{v:.13g}") for v in st.chi()]
            print(f"E={E:g}: {m} steps done after {time.perf_counter() - t0:.0f} s", flush=True)
        row["logsum_final"] = [float(f"{v:.13g}") for v in st.logsum]
        row["dE_max_final"] = [float(f"{v:.4g}") for v in st.dE_max]
        rec["energies"][f"{E:g}"] = row
    _write(rec, out)


def _merge_base(rec, out):
    """The existing record at out, checked to describe the same cells and marks
    as rec, so that energies run now can be added to it."""
    if not os.path.exists(out):
        return rec
    with open(out) as f:
        old = json.load(f)
    for key in ("grid", "eps", "h", "renorm_every", "scheme", "seed", "sample_seed", "cells",
                "cells_sha256", "marks"):
        if old.get(key) != rec[key]:
            raise SystemExit(f"{out}: {key} is {old.get(key)!r}, this run has {rec[key]!r}")
    return old


def _write(rec, out):
    tmp = out + ".tmp"
    with open(tmp, "w") as f:
        json.dump(rec, f, separators=(",", ":"))
    os.replace(tmp, out)
    print("wrote", out)


def run_ulp(args, idx):
    rec = {"what": "oracle chi_t from initial angles moved up by one ulp (np.nextafter) on the sampled cells; "
                   "written by tests/golden/make_oracle_scan_1e6.py --ulp from oracle/ only",
           "grid": G, "eps": EPS, "h": H, "renorm_every": R, "scheme": "yoshida6a", "seed": SEED,
           "sample_seed": SAMPLE_SEED, "cells": len(idx),
           "cells_sha256": hashlib.sha256(idx.astype("<i8").tobytes()).hexdigest(),
           "marks": list(MARKS), "energies": {}}
    out = args.out or OUT_ULP
    rec = _merge_base(rec, out)
    for E in args.ulp:
        X, P = initial_state(E, idx, ulp=True)
        st = oracle.State(X, P, oracle.Params(eps=EPS, h=H, renorm_every=R))
        row = {"chi": {}}
        t0 = time.perf_counter()
        for m in MARKS:
            while st.steps < m:
                st.advance(min(100_000, m - st.steps), threads=args.threads)
            row["chi"][str(m)] = [float(f"{v:.13g}") for v in st.chi()]
            print(f"E={E:g} (one ulp): {m} steps done after {time.perf_counter() - t0:.0f} s", flush=True)
        rec["energies"][f"{E:g}"] = row
    _write(rec, out)


if __name__ == "__main__":
    main()
