"""Pins of the oracle's MEGNO (mean exponential growth factor of nearby orbits,
Cincotta & Simo 2000), the alternative tangent-based indicator next to the
FTLE.  The paper defines no indicator of this kind; what pins the oracle here
is (1) the free flow (eps = 0, Sec. II), where the tangent norm is known in
closed form; (2) the limits the theory fixes: <Y> -> 0 on a stable periodic
orbit, -> 2 under linear tangent growth, ~ lambda t / 2 under exponential
growth; (3) the Abel-summation identity tying Y to the history of the
renormalisation log sum, which is itself pinned by the FTLE tests.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs

TWO_PI = 2.0 * math.pi


def _free_closed_form(m: int, dt: float):
    """eps = 0, w0 = (1, ..., 1)/sqrt 6: dX(t) = dX0 + t dP0, dP = dP0, so
    |w(t)|^2 = ((1 + t)^2 + 1) / 2 and renormalisation does not change the
    growth of a linear flow over one interval."""
    t = dt * np.arange(m + 1)
    lnN = 0.5 * np.log(((1.0 + t) ** 2 + 1.0) / 2.0)
    l = np.diff(lnN)                                  # growth logs of intervals 1..m
    j = np.arange(1, m + 1)
    Y = 2.0 * np.cumsum(j * l) / j                    # Y_1 .. Y_m
    return Y[-1], np.cumsum(Y)[-1] / m


@pytest.mark.parametrize("R,m", [(1, 7), (10, 50), (7, 13)])
def test_megno_free_flow_closed_form(R, m):
    prm = oracle.Params(eps=0.0, renorm_every=R)
    X = inputs.angles(0, np.arange(15, dtype=np.uint64)).reshape(3, 5)
    P = np.array([[1.3, -0.2, 7.0, 0.0, 2.5], [0.4, 3.3, -1.0, 0.0, 2.5], [2.0, 0.1, 0.5, 0.0, -9.0]])
    st = oracle.State(X, P, prm).advance(R * m + (R - 1))   # a partial interval does not count
    y_ref, ym_ref = _free_closed_form(m, R * prm.h)
    assert st.renorm_count() == m
    np.testing.assert_allclose(st.megno_y(), y_ref, rtol=1e-12)
    np.testing.assert_allclose(st.megno_mean(), ym_ref, rtol=1e-12)


def test_megno_linear_growth_tends_to_two():
    """Quasi-periodic (here: free) motion, |w| ~ t: <Y> -> 2, with an error that falls
    roughly like (ln m)^2 / m."""
    prm = oracle.Params(eps=0.0, renorm_every=1)
    X = np.full((3, 1), 0.3)
    P = np.array([[1.0], [2.0], [3.0]])
    st = oracle.State(X, P, prm)
    err = []
    for m in (2000, 18000):
        st.advance(m)
        err.append(abs(st.megno_mean()[0] - 2.0))
    assert err[1] < 0.05 and err[1] < 0.3 * err[0], err
    assert abs(st.megno_y()[0] - 2.0) < 0.02


def test_megno_stable_equilibrium_tends_to_zero():
    """(x, y, z) = (pi, 0, 0), P = 0 minimises Hp (Hessian diag(2, 2, 4) at eps = 1): the
    tangent map is a bounded rotation and <Y> -> 0."""
    prm = oracle.Params(eps=1.0, renorm_every=5)
    X = np.array([[math.pi], [0.0], [0.0]])
    P = np.zeros((3, 1))
    st = oracle.State(X, P, prm).advance(20000)
    assert abs(st.megno_mean()[0]) < 0.02
    # the tangent stays bounded, so the FTLE goes to zero as well
    assert abs(st.chi()[0]) < 0.01


def test_megno_abel_identity_against_logsum_history():
    """Y_m = (2/m) sum_j j l_j = 2 L_m - (2/m) sum_{k<m} L_k with L_k the log sum after k
    renormalisations (summation by parts); <Y>_m = (1/m) sum Y_k.  Checked on chaotic
    and regular trajectories with the log sum read after every interval."""
    E = 15.0
    prm = oracle.Params(eps=1.0, renorm_every=20)
    rng = np.random.default_rng(3)
    n = 6
    X = rng.uniform(0, TWO_PI, (3, n))
    P = np.zeros((3, n))
    P[0] = P[1] = math.sqrt(E) + rng.normal(0, 0.01, n)
    P[2] = rng.uniform(-1, 1, n)
    st = oracle.State(X, P, prm)
    L = [np.zeros(n)]
    for _ in range(300):
        st.advance(prm.renorm_every)
        L.append(st.logsum.copy())
    L = np.array(L)                        # L[k] after k renormalisations
    m = len(L) - 1
    Ys = np.array([2.0 * L[k] - 2.0 / k * L[:k].sum(axis=0) for k in range(1, m + 1)])
    np.testing.assert_allclose(st.megno_y(), Ys[-1], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(st.megno_mean(), Ys.mean(axis=0), rtol=1e-10, atol=1e-10)


def test_megno_slope_matches_ftle_on_chaotic_orbits():
    """Exponential growth at rate lambda gives <Y> ~ lambda t / 2: on orbits the FTLE
    classifies as chaotic, 2 <Y> / t is within 35 % of chi (both finite-time)."""
    E = 15.0
    prm = oracle.Params(eps=1.0, renorm_every=100)
    rng = np.random.default_rng(7)
    n = 8
    X = rng.uniform(0, TWO_PI, (3, n))
    P = np.zeros((3, n))
    P[0] = P[1] = math.sqrt(E)
    P[2] = rng.uniform(-0.5, 0.5, n)
    st = oracle.State(X, P, prm).advance(100000)
    chaotic = st.classify().astype(bool)
    assert chaotic.sum() >= 3
    t = st.time()
    ratio = 2.0 * st.megno_mean()[chaotic] / t / st.chi()[chaotic]
    assert np.all(np.abs(ratio - 1.0) < 0.35), ratio
    assert np.all(st.megno_mean()[chaotic] > 20.0)
