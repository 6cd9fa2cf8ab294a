"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module holds none of the method's arithmetic: it only draws counter-based
random numbers and lays out grids and boxes of initial conditions.  The
fixed-energy p_z (which needs the potential of Eq. 2) is computed by each side
on its own.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), counter form: output k of the stream seeded
with s is mix(s + (k + 1) * gamma), gamma = 0x9E3779B97F4A7C15, with the
published 64-bit finaliser (shift 30 / 27 / 31, multipliers 0xBF58476D1CE4E5B9
and 0x94D049BB133111EB).  Trajectory t of a grid draws its three angles from
counters 3t, 3t+1, 3t+2; trajectory t of a box draws counters 6t .. 6t+5.
A uniform double in [0, 1) is (r >> 11) * 2^-53, an angle is that times 2 pi.
The GPU initial-condition kernel draws the same counters, so both sides see
bit-identical angles and grids.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
TWO_PI = 6.283185307179586476925286766559
INV_2_53 = 1.0 / 9007199254740992.0


def splitmix64(seed: int, counters) -> np.ndarray:
    """Output number `counters` (0-based) of the SplitMix64 stream seeded with `seed`."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(r: np.ndarray) -> np.ndarray:
    """53-bit uniform double in [0, 1)."""
    return (r >> np.uint64(11)).astype(np.float64) * INV_2_53


def angles(seed: int, counters) -> np.ndarray:
    """Uniform angle in [0, 2 pi) (the torus of Sec. IV)."""
    return uniform01(splitmix64(seed, counters)) * TWO_PI


def grid_halfwidth(E: float, eps: float) -> float:
    """Half-width a of the (p_x, p_y) grid: a = 0.9 sqrt(E - 2|eps|), so that the
    fixed-energy p_z^2 = 2(E - eps Hp) - p_x^2 - p_y^2 stays positive (|Hp| <= 2)."""
    if E <= 2.0 * abs(eps):
        raise ValueError("grid slice needs E > 2|eps|")
    return 0.9 * math.sqrt(E - 2.0 * abs(eps))


def grid_slice(G: int, E: float, eps: float = 1.0, seed: int = 0, rows: tuple[int, int] | None = None):
    """2-D slice of initial actions: G x G grid over (p_x, p_y) in [-a, a]^2 (cell
    centres), angles uniform from `seed`.  Trajectory t = j * G + i has
    p_x from column i and p_y from row j.  Returns (X[3][n], Pxy[2][n]); p_z
    is left to the fixed-energy step.  `rows` = (j0, j1) selects a band of rows
    (a shard)."""
    a = grid_halfwidth(E, eps)
    j0, j1 = (0, G) if rows is None else rows
    t = np.arange(j0 * G, j1 * G, dtype=np.int64)
    i = t % G
    j = t // G
    ui = (i.astype(np.float64) + 0.5) / float(G)
    uj = (j.astype(np.float64) + 0.5) / float(G)
    px = (2.0 * ui - 1.0) * a
    py = (2.0 * uj - 1.0) * a
    c = 3 * t.astype(np.uint64)
    X = np.stack([angles(seed, c), angles(seed, c + np.uint64(1)), angles(seed, c + np.uint64(2))])
    return X, np.stack([px, py])


def box(n: int, lo=(10.0, 4.0, 25.0), hi=(11.0, 5.0, 26.0), seed: int = 0, offset: int = 0):
    """Uniform box: X ~ U[0, 2pi)^3, P ~ U(prod [lo_a, hi_a)).  Returns (X, P)."""
    t = np.arange(offset, offset + n, dtype=np.uint64)
    c = np.uint64(6) * t
    X = np.stack([angles(seed, c + np.uint64(k)) for k in range(3)])
    P = np.stack([lo[k] + (hi[k] - lo[k]) * uniform01(splitmix64(seed, c + np.uint64(3 + k))) for k in range(3)])
    return X, P


def sample_cells(n_total: int, k: int, seed: int = 12345) -> np.ndarray:
    """k distinct trajectory indices of [0, n_total), sorted (seeded subset)."""
    if k >= n_total:
        return np.arange(n_total, dtype=np.int64)
    r = (splitmix64(seed, np.arange(8 * k + 64, dtype=np.uint64)) % np.uint64(n_total)).astype(np.int64)
    _, first = np.unique(r, return_index=True)
    picked = r[np.sort(first)]
    if len(picked) < k:
        raise ValueError("sample_cells: too few distinct draws")
    return np.sort(picked[:k])


def sphere_directions(n: int, seed: int = 0, cos_range=(-1.0, 1.0), phi_range=(0.0, TWO_PI), offset: int = 0):
    """Angles uniform on the torus and momentum directions uniform on a patch of
    the unit sphere (cos theta uniform in cos_range, phi uniform in phi_range):
    the ensembles of Sec. IV, Figs. 2-3 (whole sphere, or a segment for zooms).
    Trajectory t draws counters 5t .. 5t+4.  Returns (X[3][n], nhat[3][n]);
    the modulus of P is left to the fixed-energy step."""
    t = np.arange(offset, offset + n, dtype=np.uint64)
    c = np.uint64(5) * t
    X = np.stack([angles(seed, c + np.uint64(k)) for k in range(3)])
    u = uniform01(splitmix64(seed, c + np.uint64(3)))
    w = uniform01(splitmix64(seed, c + np.uint64(4)))
    ct = cos_range[0] + (cos_range[1] - cos_range[0]) * u
    ph = phi_range[0] + (phi_range[1] - phi_range[0]) * w
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    return X, np.stack([st * np.cos(ph), st * np.sin(ph), ct])


def gaussian_velocities(n: int, center=(0.0, 0.0), sigma: float = 0.01, seed: int = 0, offset: int = 0):
    """Angles uniform on the torus, (p_x, p_y) Gaussian about `center` with
    standard deviation sigma (Box-Muller on two SplitMix64 uniforms; the
    ensemble of Fig. 4).  Counters 5t .. 5t+4.  Returns (X[3][n], Pxy[2][n]);
    p_z is left to the fixed-energy step."""
    t = np.arange(offset, offset + n, dtype=np.uint64)
    c = np.uint64(5) * t
    X = np.stack([angles(seed, c + np.uint64(k)) for k in range(3)])
    u1 = 1.0 - uniform01(splitmix64(seed, c + np.uint64(3)))       # (0, 1]
    u2 = uniform01(splitmix64(seed, c + np.uint64(4)))
    r = np.sqrt(-2.0 * np.log(u1))
    return X, np.stack([center[0] + sigma * r * np.cos(TWO_PI * u2), center[1] + sigma * r * np.sin(TWO_PI * u2)])
