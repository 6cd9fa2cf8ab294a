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
