"""Oracle for the Arnold-web ensemble propagator -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 CPU implementation of what the GPU hot path computes: the
C core (``arnold_oracle.c``) iterates the map, and this module adds the
per-trajectory indicators and ensemble statistics in plain numpy.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline and
reference legs may import it; the product package never does, and this module
imports nothing from the product package.

Every function cites the passage of the paper (arXiv:1107.4107) it follows.
Readings adopted where the paper is silent:
  * chaos indicator: finite-time Lyapunov exponent chi_t = ln(|w(t)| / |w(0)|) / t
    of the tangent map (the paper names FTLEs as the competing indicator,
    Sec. V), w(0) = (1, ..., 1) / sqrt(6), t = steps * h;
  * classification: chaotic iff chi_t > kappa * ln(max(t, e)) / t, kappa = 10
    (regular orbits have linearly growing tangents, chi_t ~ ln t / t);
  * the paper's own indicator is V = [X(t + dt) - X(t)] / dt with unwrapped
    angles (Sec. IV); dt = whole run when window = 0.
Parity of the statistics (histogram of log10 chi, chaotic fraction, moments)
is pinned by brute-force recounting in the tests; nothing here is unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "arnold_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
TWO_PI = 6.283185307179586476925286766559

SCHEMES = {"yoshida6a": 0, "triplejump6": 1, "leapfrog2": 2}


def build(force: bool = False) -> str:
    """Compile the C oracle (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("h", ctypes.c_double), ("scheme", ctypes.c_int32),
                ("renorm_every", ctypes.c_int32), ("window", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        L.oracle_run.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 dp, dp, dp, ip, dp, dp, dp, dp, dp, dp]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_energy.argtypes = [ctypes.c_double, ctypes.c_int64, dp, dp, dp]
        L.oracle_pz_from_energy.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64, dp, dp]
        L.oracle_pz_from_energy.restype = ctypes.c_int64
        L.oracle_momenta_on_shell.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64, dp, dp, dp]
        L.oracle_momenta_on_shell.restype = ctypes.c_int64
        L.oracle_track.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                   ctypes.POINTER(ctypes.c_uint8)]
        L.oracle_track.restype = ctypes.c_int
        L.oracle_jacobian.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp, dp]
        L.oracle_jacobian.restype = ctypes.c_int
        L.oracle_scheme_weights.argtypes = [ctypes.c_int, dp]
        L.oracle_scheme_weights.restype = ctypes.c_int
        L.oracle_hp.argtypes = [ctypes.c_double] * 3
        L.oracle_hp.restype = ctypes.c_double
        L.oracle_grad_hp.argtypes = [dp, dp]
        L.oracle_hess_hp.argtypes = [dp, dp]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if a.dtype == np.int64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    raise TypeError(a.dtype)


@dataclass
class Params:
    """Map parameters: eps of Eq. 1, step h (Sec. III), scheme, R, window W."""
    eps: float = 1.0
    h: float = 0.02 * math.pi
    scheme: str = "yoshida6a"
    renorm_every: int = 100
    window: int = 0

    def c(self):
        return _Params(self.eps, self.h, SCHEMES[self.scheme], self.renorm_every, self.window)


def scheme_weights(scheme: str) -> np.ndarray:
    w = np.zeros(9)
    m = lib().oracle_scheme_weights(SCHEMES[scheme], _ptr(w))
    return w[:m].copy()


def hp(x, y, z) -> float:
    """Eq. 2."""
    return lib().oracle_hp(float(x), float(y), float(z))


def grad_hp(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    g = np.zeros(3)
    lib().oracle_grad_hp(_ptr(X), _ptr(g))
    return g


def hess_hp(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    H = np.zeros(9)
    lib().oracle_hess_hp(_ptr(X), _ptr(H))
    return H.reshape(3, 3)


def energy(eps: float, X: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Eq. 1 for SoA arrays X[3][n], P[3][n]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = X.shape[1]
    E = np.zeros(n)
    lib().oracle_energy(eps, n, _ptr(X), _ptr(P), _ptr(E))
    return E


def pz_from_energy(E: float, eps: float, X: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Fixed-energy p_z (Sec. IV, Fig. 4 caption).  Returns a new P."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    lib().oracle_pz_from_energy(E, eps, X.shape[1], _ptr(X), _ptr(P))
    return P


def momenta_on_shell(E: float, eps: float, X: np.ndarray, nhat: np.ndarray) -> np.ndarray:
    """P = sqrt(2 (E - eps Hp(X))) nhat (Sec. IV: ensembles on the sphere S)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    nhat = np.ascontiguousarray(nhat, dtype=np.float64)
    P = np.zeros_like(nhat)
    lib().oracle_momenta_on_shell(E, eps, X.shape[1], _ptr(X), _ptr(nhat), _ptr(P))
    return P


def track_patch(params: Params, X, P, n_steps: int, patch, step0: int = 0):
    """Area tracking (Sec. IV): returns (X_N, P_N, left[n] uint8) with left = 1 for
    trajectories whose momentum direction left the patch (cos_lo, cos_hi,
    phi_lo, phi_hi) at any sample (every renorm_every steps)."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    n = X.shape[1]
    left = np.zeros(n, dtype=np.uint8)
    pa = np.ascontiguousarray(patch, dtype=np.float64)
    rc = lib().oracle_track(ctypes.byref(params.c()), n, step0, n_steps, _ptr(X), _ptr(P), _ptr(pa),
                            left.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError("oracle_track rejected its arguments")
    return X, P, left


def velocity_histogram(V: np.ndarray, n_cos: int, n_phi: int, patch=(-1.0, 1.0, 0.0, TWO_PI), keep=None) -> np.ndarray:
    """Counts of the direction of V (Sec. IV: the density F of V projected on the
    sphere S) in n_cos x n_phi cells of equal width in cos theta and phi over
    the patch; directions outside the patch, and trajectories with keep = 0,
    are not counted."""
    V = np.asarray(V, dtype=np.float64)
    m = np.sqrt(V[0] ** 2 + V[1] ** 2 + V[2] ** 2)
    c = V[2] / m
    phi = np.arctan2(V[1], V[0])
    phi = np.where(phi < 0.0, phi + TWO_PI, phi)
    counts = np.zeros((n_cos, n_phi), dtype=np.int64)
    for i in range(V.shape[1]):
        if keep is not None and not keep[i]:
            continue
        if not (patch[0] <= c[i] <= patch[1] and patch[2] <= phi[i] <= patch[3]):
            continue
        a = min(int((c[i] - patch[0]) / (patch[1] - patch[0]) * n_cos), n_cos - 1)
        b = min(int((phi[i] - patch[2]) / (patch[3] - patch[2]) * n_phi), n_phi - 1)
        counts[a, b] += 1
    return counts


class State:
    """Per-trajectory state of the ensemble (SoA, FP64)."""

    def __init__(self, X, P, params: Params, tangent: bool = True, W=None):
        self.X = np.array(X, dtype=np.float64, order="C", copy=True)
        self.P = np.array(P, dtype=np.float64, order="C", copy=True)
        n = self.X.shape[1]
        self.n = n
        self.params = params
        if tangent:
            self.W = (np.full((6, n), 1.0 / math.sqrt(6.0)) if W is None
                      else np.array(W, dtype=np.float64, order="C", copy=True))
        else:
            self.W = None
        self.lap = np.zeros((3, n), dtype=np.int64)
        self.xref = self.X.copy()
        self.logsum = np.zeros(n)
        self.dE_max = np.zeros(n)
        self.e0 = energy(params.eps, self.X, self.P)
        self.P0 = self.P.copy()
        self.V = np.zeros((3, n))
        self.megno = np.zeros((2, n)) if tangent else None   # (S, Ysum), see megno_mean()
        self.steps = 0

    def run(self, n_steps: int, lo: int = 0, hi: int | None = None) -> "State":
        """Composite steps (Sec. III) on trajectories [lo, hi); ranges of one state
        may run concurrently from threads (ctypes releases the GIL)."""
        hi = self.n if hi is None else hi
        if hi <= lo:
            return self
        sl = slice(lo, hi)
        X = np.ascontiguousarray(self.X[:, sl])
        P = np.ascontiguousarray(self.P[:, sl])
        W = None if self.W is None else np.ascontiguousarray(self.W[:, sl])
        lap = np.ascontiguousarray(self.lap[:, sl])
        xref = np.ascontiguousarray(self.xref[:, sl])
        logsum = np.ascontiguousarray(self.logsum[sl])
        dE = np.ascontiguousarray(self.dE_max[sl])
        e0 = np.ascontiguousarray(self.e0[sl])
        V = np.ascontiguousarray(self.V[:, sl])
        mg = None if self.megno is None else np.ascontiguousarray(self.megno[:, sl])
        rc = lib().oracle_run(ctypes.byref(self.params.c()), hi - lo, self.steps, n_steps,
                              _ptr(X), _ptr(P), _ptr(W), _ptr(lap), _ptr(xref), _ptr(logsum),
                              _ptr(dE), _ptr(e0), _ptr(V), _ptr(mg))
        if rc != 0:
            raise ValueError("oracle_run rejected its arguments")
        self.X[:, sl] = X
        self.P[:, sl] = P
        if W is not None:
            self.W[:, sl] = W
        self.lap[:, sl] = lap
        self.xref[:, sl] = xref
        self.logsum[sl] = logsum
        self.dE_max[sl] = dE
        self.V[:, sl] = V
        if mg is not None:
            self.megno[:, sl] = mg
        return self

    def advance(self, n_steps: int, threads: int = 1) -> "State":
        """Run every trajectory n_steps and bump the step counter."""
        if threads <= 1:
            self.run(n_steps)
        else:
            from concurrent.futures import ThreadPoolExecutor
            edges = np.linspace(0, self.n, threads + 1).astype(int)
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda k: self.run(n_steps, edges[k], edges[k + 1]), range(threads)))
        self.steps += n_steps
        return self

    # ---- indicators (Sec. IV and the FTLE reading) ----
    def time(self) -> float:
        return self.steps * self.params.h

    def unwrapped_displacement(self) -> np.ndarray:
        """X(t) - X(window start) with laps restored (Sec. IV: V uses unwrapped X)."""
        return self.X - self.xref + TWO_PI * self.lap

    def chi(self) -> np.ndarray:
        """FTLE chi_t = (sum of renormalisation logs + ln|w|) / t."""
        return (self.logsum + np.log(np.sqrt(np.sum(self.W * self.W, axis=0)))) / self.time()

    def renorm_count(self) -> int:
        """Renormalisations so far (the MEGNO sample index m)."""
        return self.steps // self.params.renorm_every

    def megno_y(self) -> np.ndarray:
        """MEGNO Y_m = (2/m) sum_j j l_j at the last renormalisation (0 before the first)."""
        m = self.renorm_count()
        return 2.0 * self.megno[0] / m if m else np.zeros(self.n)

    def megno_mean(self) -> np.ndarray:
        """Mean MEGNO <Y>_m = (1/m) sum_k Y_k: tends to 0 on stable periodic orbits, to 2 on
        quasi-periodic ones (linear tangent growth), grows like lambda t / 2 on chaotic ones."""
        m = self.renorm_count()
        return self.megno[1] / m if m else np.zeros(self.n)

    def velocity(self) -> np.ndarray:
        """Finite-time averaged velocity V = [X(t+dt) - X(t)] / dt (Sec. IV)."""
        if self.params.window > 0:
            return self.V.copy()
        return self.unwrapped_displacement() / self.time()

    def velocity_deviation(self) -> np.ndarray:
        """|V - P(0)|: Sec. IV reads a regular trajectory by its averaged velocity
        staying close to its initial momentum vector; this is that distance."""
        return np.sqrt(np.sum((self.velocity() - self.P0) ** 2, axis=0))

    def dE(self) -> np.ndarray:
        """Energy error |E(t) - E(0)| (Sec. III)."""
        return np.abs(energy(self.params.eps, self.X, self.P) - self.e0)

    def classify(self, kappa: float = 10.0) -> np.ndarray:
        return classify(self.chi(), self.time(), kappa)


def chaos_threshold(t: float, kappa: float = 10.0) -> float:
    """Regular orbits have chi_t ~ ln(t) / t; threshold kappa * ln(max(t, e)) / t."""
    return kappa * math.log(max(t, math.e)) / t


def classify(chi: np.ndarray, t: float, kappa: float = 10.0) -> np.ndarray:
    return (chi > chaos_threshold(t, kappa)).astype(np.uint8)


HIST_BINS = 200
HIST_LO = -8.0
HIST_HI = 1.0


def stats(chi: np.ndarray, dE: np.ndarray, P: np.ndarray, t: float, kappa: float = 10.0) -> dict:
    """Ensemble statistics: histogram of log10 chi over [-8, 1] in 200 bins
    (under/overflow counted apart; chi <= 0 counts as underflow), chaotic
    count, max dE, mean and population variance of each momentum component
    (F of Sec. IV is an ensemble statistic of the same kind)."""
    chi = np.asarray(chi, dtype=np.float64)
    counts = np.zeros(HIST_BINS, dtype=np.int64)
    under = over = 0
    scale = HIST_BINS / (HIST_HI - HIST_LO)
    for c in chi:
        if not (c > 0.0):
            under += 1
            continue
        u = (math.log10(c) - HIST_LO) * scale
        if u < 0.0:
            under += 1
        elif u >= HIST_BINS:
            over += 1
        else:
            counts[int(math.floor(u))] += 1
    thr = chaos_threshold(t, kappa)
    return {
        "hist": counts, "under": under, "over": over,
        "chaotic": int(np.sum(chi > thr)),
        "dE_max": float(np.max(dE)) if len(dE) else 0.0,
        "p_mean": np.mean(P, axis=1), "p_var": np.var(P, axis=1),
    }


# ---- gradient reference for the adjoint (derivatives of the N-step map) ----
def loss_variance(P: np.ndarray) -> float:
    """L = (1/3) sum_alpha Var_i P_alpha^i (population variance)."""
    return float(np.mean(np.var(P, axis=1)))


def dloss_dp(P: np.ndarray) -> np.ndarray:
    n = P.shape[1]
    return (2.0 / 3.0) * (P - P.mean(axis=1, keepdims=True)) / n


def jacobian(params: Params, X, P, n_steps: int):
    """Forward-mode derivatives of the n_steps map: returns (X_N, P_N, J[n,6,6],
    dz/dh [n,6], dz/deps [n,6])."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    P = np.array(P, dtype=np.float64, order="C", copy=True)
    n = X.shape[1]
    J = np.zeros((n, 6, 6))
    dh = np.zeros((n, 6))
    de = np.zeros((n, 6))
    rc = lib().oracle_jacobian(ctypes.byref(params.c()), n, n_steps, _ptr(X), _ptr(P), _ptr(J), _ptr(dh), _ptr(de))
    if rc != 0:
        raise ValueError("oracle_jacobian rejected its arguments")
    return X, P, J, dh, de


def gradient(params: Params, X, P, n_steps: int, dL_dxN=None, dL_dpN=None, lossfn=None):
    """Gradient of a loss of the final state w.r.t. (X0, P0, h, eps) by forward-mode
    Jacobian products (no reverse sweep).  If dL_dpN is None, the variance loss
    is used.  Returns (g_x0[3][n], g_p0[3][n], g_h, g_eps, X_N, P_N)."""
    XN, PN, J, dh, de = jacobian(params, X, P, n_steps)
    n = XN.shape[1]
    lx = np.zeros((3, n)) if dL_dxN is None else np.asarray(dL_dxN, dtype=np.float64)
    lp = dloss_dp(PN) if dL_dpN is None else np.asarray(dL_dpN, dtype=np.float64)
    lam = np.concatenate([lx, lp], axis=0).T          # [n, 6]
    g0 = np.einsum("nr,nrc->nc", lam, J)               # [n, 6]
    g_h = float(np.sum(lam * dh))
    g_e = float(np.sum(lam * de))
    return g0[:, :3].T.copy(), g0[:, 3:].T.copy(), g_h, g_e, XN, PN
