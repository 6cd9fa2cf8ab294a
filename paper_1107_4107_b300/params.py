"""Parameter plumbing between the paper's (eps, E, h) and the map's (K, eps_eff).

* Eq. 1: H = P^2/2 + eps Hp(X); the paper sets eps = 1 and lets the energy E
  control the perturbation, eps_eff = max|Hp| / E = 2/E (Eq. 3; with general
  eps, 2 eps / E).
* Sec. III: h = 1e-2 T with T = 2 pi.
* One drift-kick-drift substep of the map, in scaled momentum q = h P, reads
  q' = q - K grad Hp(X), X' = X + q' with K = eps h^2 (the "kick strength").
* Scaling P -> sqrt(eps) P', t -> t / sqrt(eps) maps (eps, E, h) onto
  (1, E / eps, sqrt(eps) h), so (K, eps_eff) fix the map up to that scaling.
"""
from __future__ import annotations

import math

TWO_PI = 2.0 * math.pi
T_PERIOD = TWO_PI          # Sec. III: T = 2 pi


def paper_h() -> float:
    """Sec. III: h = 1e-2 T."""
    return 1e-2 * T_PERIOD


def eps_eff(E: float, eps: float = 1.0) -> float:
    """Eq. 3: eps_eff = max|eps Hp| / E = 2 eps / E."""
    return 2.0 * eps / E


def energy_for(eps_eff_value: float, eps: float = 1.0) -> float:
    """Inverse of Eq. 3."""
    return 2.0 * eps / eps_eff_value


def kick_strength(eps: float, h: float) -> float:
    """K = eps h^2 of the scaled-momentum substep."""
    return eps * h * h


def h_for(K: float, eps: float = 1.0) -> float:
    return math.sqrt(K / eps)


def grads_K_eps(g_h: float, g_eps: float, h: float, eps: float) -> tuple[float, float]:
    """Chain rule from (dL/dh at fixed eps, dL/deps at fixed h) to
    (dL/dK at fixed eps, dL/deps at fixed K), with h = sqrt(K / eps)."""
    dh_dK = 1.0 / (2.0 * eps * h)          # dh/dK |_eps
    dh_deps = -h / (2.0 * eps)             # dh/deps |_K
    return g_h * dh_dK, g_eps + g_h * dh_deps


def batch_sets(seed: int = 0, n_eps: int = 8, n_K: int = 8, eps_eff_range=(1e-5, 1e-1),
               K_range=((0.005 * T_PERIOD) ** 2, (0.02 * T_PERIOD) ** 2), size_range=(1e3, 1e6),
               steps_range=(1e4, 1e6), step_scale: float = 1.0, eps: float = 1.0) -> list[dict]:
    """Parameter sets of the batched scan: an n_eps x n_K log grid of
    (eps_eff, K) -> (E = 2 eps / eps_eff, h = sqrt(K / eps)); ensemble sizes
    log-uniform in size_range (as G x G grids) and step counts log-uniform in
    steps_range (times step_scale), drawn from SplitMix64(seed)."""
    from .inputs import splitmix64, uniform01
    import numpy as np
    ee = np.geomspace(eps_eff_range[0], eps_eff_range[1], n_eps)
    KK = np.geomspace(K_range[0], K_range[1], n_K)
    m = n_eps * n_K
    u = uniform01(splitmix64(seed, np.arange(2 * m, dtype=np.uint64))).reshape(2, m)
    sizes = np.exp(np.log(size_range[0]) + u[0] * (np.log(size_range[1]) - np.log(size_range[0])))
    steps = np.exp(np.log(steps_range[0]) + u[1] * (np.log(steps_range[1]) - np.log(steps_range[0])))
    out = []
    k = 0
    for a in ee:
        for K in KK:
            G = max(8, int(round(math.sqrt(sizes[k]))))
            out.append({"eps": eps, "h": h_for(K, eps), "E": energy_for(a, eps), "G": G,
                        "n_steps": max(1, int(round(steps[k] * step_scale))), "seed": seed + k,
                        "eps_eff": float(a), "K": float(K)})
            k += 1
    return out
