"""Helpers shared by the GPU parity tests: run the same seeded inputs through the
CUDA path (C ABI via the binding) and the oracle, and measure the differences."""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_1107_4107_b300 import inputs

TWO_PI = 2.0 * math.pi


def oracle_params(eps=1.0, h=None, scheme="yoshida6a", R=100, window=0):
    return oracle.Params(eps=eps, h=0.02 * math.pi if h is None else h, scheme=scheme, renorm_every=R, window=window)


def oracle_grid_state(G, E, prm, rows=None, seed=0, cells=None):
    """The oracle's own fixed-energy grid initial conditions (Sec. IV)."""
    X, Pxy = inputs.grid_slice(G, E, prm.eps, seed=seed, rows=rows)
    if cells is not None:
        X, Pxy = X[:, cells].copy(), Pxy[:, cells].copy()
    P = np.zeros((3, X.shape[1]))
    P[:2] = Pxy
    P = oracle.pz_from_energy(E, prm.eps, X, P)
    return oracle.State(X, P, prm)


def rel_err(a, b):
    """max |a - b| / (1 + |b|) (relative for large values, absolute near zero)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / (1.0 + np.abs(b)))) if a.size else 0.0


def angle_dist(a, b):
    d = np.mod(np.asarray(a) - np.asarray(b), TWO_PI)
    return np.minimum(d, TWO_PI - d)


def compare_state(ens, st, tangent=True):
    """Per-quantity relative errors of the CUDA ensemble against the oracle state."""
    out = {}
    dX = ens.indicator("dX")
    out["dX"] = rel_err(dX, st.unwrapped_displacement())
    out["X"] = float(np.max(angle_dist(ens.indicator("X"), st.X)))
    out["P"] = rel_err(ens.indicator("P"), st.P)
    if tangent:
        W = ens.indicator("tangent")
        out["tangent"] = rel_err(W, st.W)
        if st.steps > 0:
            out["chi"] = rel_err(ens.indicator("chi"), st.chi())
    if st.steps > 0:
        out["V"] = rel_err(ens.indicator("V"), st.velocity())
    out["dE_max"] = float(np.max(np.abs(ens.indicator("dE_max") - st.dE_max)))
    return out


def cell_growth(st):
    """Each cell's own tangent growth exp(chi t) over the run, from the oracle (at
    least 1): the first-order amplification of an error made along the way."""
    return np.maximum(1.0, np.exp(np.minimum(st.chi() * st.time(), 700.0)))


def growth_scaled(got, ref, growth, bound, power=1):
    """Per-cell parity bar: |got - ref| / (1 + |ref|) (worst component of a
    [k][n] quantity) <= bound * growth^power, for every cell.  power = 1 for the
    state, V and the FTLE (first-order propagation of rounding); power = 2 for
    the tangent components, which are first derivatives of the flow and so
    carry the second-order sensitivity of the state errors.  Returns
    (ok, worst err / bar)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref) / (1.0 + np.abs(ref))
    if err.ndim == 2:
        err = np.max(err, axis=0)
    bar = bound * np.asarray(growth, dtype=np.float64) ** power
    return bool(np.all(err <= bar)), float(np.max(err / bar))


def advance_with_growth_history(st, n_steps, threads=1):
    """Advance the oracle state n_steps (a multiple of its renormalisation
    interval R) and return each cell's largest tangent growth over any
    sub-interval between renormalisations, max_k exp(L_k - min_{j<=k} L_j)
    (L_k the log sum after k renormalisations, L_0 = 0).  ln|w| is not monotone:
    after a chaotic transient the tangent can shrink again, so the final
    exp(chi t) can understate how much an error made along the way was
    stretched; this maximum does not."""
    R = st.params.renorm_every
    if n_steps % R:
        raise ValueError("n_steps must be a multiple of the renormalisation interval")
    L0 = st.logsum.copy()
    low = L0.copy()
    best = np.zeros(st.n)
    for _ in range(n_steps // R):
        st.advance(R, threads=threads)
        low = np.minimum(low, st.logsum)
        best = np.maximum(best, st.logsum - low)
    return np.exp(np.minimum(best, 700.0))
