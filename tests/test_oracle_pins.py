"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the mistake it would catch.  None of them re-types the
oracle's formulas: they use closed forms, a textbook map written independently,
elliptic-integral periods, invariants, convergence orders and brute force.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import ellipk

import oracle
from paper_1107_4107_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TWO_PI = 2.0 * math.pi


def _box(n, seed=3, lo=(-3.0, -2.0, -1.5), hi=(3.0, 2.0, 1.5)):
    return inputs.box(n, lo=lo, hi=hi, seed=seed)


def _unwrapped(st):
    return st.X + TWO_PI * st.lap


# ---------------------------------------------------------------- eps = 0 ---
@pytest.mark.parametrize("scheme", ["yoshida6a", "triplejump6", "leapfrog2"])
def test_free_rotation_closed_form(scheme):
    """Sec. II: at eps = 0, X(t) = X(0) + P t and P is constant.  Catches wrong
    drift coefficients (weights not summing to one step), lap/wrap mistakes,
    the V formula and the tangent drift (dX(t) = dX0 + t dP0)."""
    X, P = _box(64, lo=(-30.0, -30.0, -30.0), hi=(30.0, 30.0, 30.0))
    prm = oracle.Params(eps=0.0, h=0.0731, scheme=scheme, renorm_every=7)
    st = oracle.State(X, P, prm)
    S = 1000
    st.advance(S)
    t = S * prm.h
    assert np.array_equal(st.P, P)
    np.testing.assert_allclose(_unwrapped(st), X + P * t, rtol=0, atol=1e-11 * (1 + np.abs(P * t)).max())
    assert np.all((st.X >= 0) & (st.X < TWO_PI))
    np.testing.assert_allclose(st.velocity(), P, rtol=1e-12, atol=1e-12)
    # w0 = (1,..,1)/sqrt(6): |w(t)|^2 = (3 (1 + t)^2 + 3) / 6
    chi_exact = 0.5 * math.log((3.0 * (1.0 + t) ** 2 + 3.0) / 6.0) / t
    np.testing.assert_allclose(st.chi(), chi_exact, rtol=1e-12)
    assert st.dE().max() < 1e-10 * 30 ** 2


def test_window_velocity_closed_form():
    """Sec. IV: V over a window dt of W steps equals P exactly at eps = 0."""
    X, P = _box(16, lo=(-20.0, -20.0, -20.0), hi=(20.0, 20.0, 20.0))
    prm = oracle.Params(eps=0.0, window=50)
    st = oracle.State(X, P, prm)
    st.advance(175)
    np.testing.assert_allclose(st.V, P, rtol=1e-12)
    assert np.all(np.abs(st.lap) <= 25 * 20 * prm.h / TWO_PI + 2)


# ------------------------------------------------------- standard map pin ---
def _chirikov(theta, I, K, n):
    """Chirikov standard map I' = I + K sin(theta), theta' = theta + I' (mod 2 pi)."""
    for _ in range(n):
        I = I + K * math.sin(theta)
        theta = math.fmod(theta + I, TWO_PI)
        if theta < 0:
            theta += TWO_PI
    return theta, I


def test_leapfrog_is_standard_map_on_invariant_plane():
    """On y = p_y = z = p_z = 0, Hp = 2 cos x and the leapfrog map in (x + h p / 2, h p)
    is the Chirikov standard map with K = 2 eps h^2.  Catches a wrong force sign,
    a wrong force factor, and kick/drift order mistakes."""
    eps, h = 0.7, 0.3
    rng = np.random.default_rng(5)
    x0 = rng.uniform(0, TWO_PI, 8)
    p0 = rng.uniform(-2, 2, 8)
    X = np.zeros((3, 8)); X[0] = x0
    P = np.zeros((3, 8)); P[0] = p0
    st = oracle.State(X, P, oracle.Params(eps=eps, h=h, scheme="leapfrog2"), tangent=False)
    n = 300
    st.advance(n)
    K = 2.0 * eps * h * h
    for i in range(8):
        th, I = _chirikov(x0[i] + 0.5 * h * p0[i], h * p0[i], K, n)
        assert abs(st.P[0, i] - I / h) < 1e-9 * (1 + abs(I / h))
        d = (st.X[0, i] + 0.5 * h * st.P[0, i] - th) % TWO_PI
        assert min(d, TWO_PI - d) < 1e-9
    assert np.all(st.X[1:] == 0.0) and np.all(st.P[1:] == 0.0)


def test_invariant_subspaces_exact():
    """dHp/dy ~ sin y and dHp/dz ~ sin 2z: y = p_y = 0 and z = p_z = 0 are invariant
    (exactly, since sin 0 = 0).  Catches a force component mixing axes."""
    X, P = _box(32)
    X1, P1 = X.copy(), P.copy()
    X1[1] = 0.0; P1[1] = 0.0
    st = oracle.State(X1, P1, oracle.Params(), tangent=False).advance(200)
    assert np.all(st.X[1] == 0.0) and np.all(st.P[1] == 0.0)
    X2, P2 = X.copy(), P.copy()
    X2[2] = 0.0; P2[2] = 0.0
    st = oracle.State(X2, P2, oracle.Params(), tangent=False).advance(200)
    assert np.all(st.X[2] == 0.0) and np.all(st.P[2] == 0.0)


def test_velocity_deviation_closed_forms():
    """|V - P(0)| (Sec. IV's reading of V): 0 at eps = 0, where V = P(0) exactly;
    and for a pendulum trapped about x = pi on the invariant plane, whose x
    stays within its amplitude of pi, V_x -> 0 like 2 amp / t while P(0) = (p0,
    0, 0): |V - P(0)| -> |p0| within that bound.  Catches the momentum taken
    at the end of the run instead of the start, and a wrong norm."""
    X, P = _box(32, lo=(-20.0, -20.0, -20.0), hi=(20.0, 20.0, 20.0))
    st = oracle.State(X, P, oracle.Params(eps=0.0, h=0.05), tangent=False).advance(300)
    assert np.max(st.velocity_deviation()) < 1e-11
    eps, p0 = 1.0, 0.5
    X = np.zeros((3, 1)); X[0, 0] = math.pi + 0.3
    P = np.zeros((3, 1)); P[0, 0] = p0
    st = oracle.State(X, P, oracle.Params(eps=eps), tangent=False).advance(1000)
    # energy p^2/2 + 2 eps cos x < 2 eps: trapped; amplitude from the energy
    amp = math.acos(-(0.5 * p0 * p0 + 2.0 * eps * math.cos(math.pi + 0.3)) / (2.0 * eps))
    t = st.time()
    assert abs(abs(st.P[0, 0]) - p0) > 0.05              # |P(t)| is not |P(0)|: the reading needs P(0)
    assert abs(st.velocity_deviation()[0] - p0) <= 2.0 * amp / t


def test_pendulum_period_elliptic():
    """On the invariant plane H = p^2/2 + 2 eps cos x: a pendulum about x = pi with
    omega0^2 = 2 eps; period 4 K(k) / omega0, k = sin(amplitude / 2).  Catches a
    wrong potential amplitude or integrator mistakes that the energy hides."""
    eps = 1.0
    amp = 1.2
    h = 0.01
    X = np.zeros((3, 1)); X[0, 0] = math.pi + amp
    P = np.zeros((3, 1))
    st = oracle.State(X, P, oracle.Params(eps=eps, h=h), tangent=False)
    ps = [0.0]
    for _ in range(1200):
        st.advance(1)
        ps.append(st.P[0, 0])
    ps = np.array(ps)
    # p starts at 0 and becomes negative; upward zero crossings of p are one period apart.
    cross = [k - 1 + (-ps[k - 1]) / (ps[k] - ps[k - 1]) for k in range(1, len(ps)) if ps[k - 1] < 0 <= ps[k]]
    period = (cross[1] - cross[0]) * h
    exact = 4.0 * ellipk(math.sin(amp / 2) ** 2) / math.sqrt(2.0 * eps)
    assert abs(period - exact) < 2e-6 * exact


# ------------------------------------------------------------------ order ---
@pytest.mark.parametrize("scheme,order", [("yoshida6a", 6), ("triplejump6", 6), ("leapfrog2", 2)])
def test_convergence_order(scheme, order):
    """Sec. III: a sixth-order integrator.  Halving h at fixed t shrinks the state
    error (against an h/16 reference) by 2^order within 20 %.  Catches wrong
    composition weights or substep order."""
    X, P = _box(6, seed=11, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0))
    t_end = 2.0
    hs = [0.2, 0.1] if order == 6 else [0.02, 0.01]

    def run(h):
        n = int(round(t_end / h))
        st = oracle.State(X, P, oracle.Params(eps=1.0, h=h, scheme=scheme), tangent=False).advance(n)
        return np.concatenate([_unwrapped(st), st.P])

    ref = run(hs[-1] / 16)
    e = [np.abs(run(h) - ref).max() for h in hs]
    ratio = e[0] / e[1]
    assert abs(ratio / 2 ** order - 1) < 0.2, (e, ratio)


def test_energy_error_sixth_order_and_paper_step():
    """Sec. III quotes |E(t) - E(0)| < 1e-8 at h = 0.01 T, T = 2 pi.  The energy error
    of the map falls by ~64 per halving of h (sixth order); at E = 400 the
    paper's h gives ~1e-2, and 1e-8 is met from h = 0.01 T / 8 (recorded reading)."""
    X, Pxy = inputs.grid_slice(4, 400.0)
    P = np.zeros((3, 16)); P[:2] = Pxy
    P = oracle.pz_from_energy(400.0, 1.0, X, P)
    errs = []
    for f in (0.25, 0.125):
        st = oracle.State(X, P, oracle.Params(h=0.02 * math.pi * f, renorm_every=10), tangent=False)
        st.advance(int(round(500 / f)))
        errs.append(st.dE_max.max())
    assert 40 < errs[0] / errs[1] < 100
    assert errs[1] < 1e-8


# ----------------------------------------------------- structure of the map ---
def test_symplectic_jacobian():
    """Sec. III: the integrator is symplectic, so the step Jacobian J obeys
    J^T Omega J = Omega and det J = 1.  Catches a tangent/Hessian mistake."""
    X, P = _box(6, seed=2, lo=(-2.0, -2.0, -2.0), hi=(2.0, 2.0, 2.0))
    _, _, J, _, _ = oracle.jacobian(oracle.Params(eps=1.0, h=0.05), X, P, 100)
    Om = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])
    for k in range(J.shape[0]):
        Jk = J[k]
        s = max(1.0, np.abs(Jk).max() ** 2)
        assert np.abs(Jk.T @ Om @ Jk - Om).max() < 1e-12 * s
        assert abs(np.linalg.det(Jk) - 1.0) < 1e-10 * s


def test_tangent_matches_central_differences():
    """Brute force on tiny inputs: (Phi(z + eta e_k) - Phi(z - eta e_k)) / 2 eta vs J e_k,
    and the run's tangent vector vs J w0.  Catches Hessian entries and the
    tangent kick/drift."""
    X, P = _box(4, seed=4, lo=(-2.0, -2.0, -2.0), hi=(2.0, 2.0, 2.0))
    prm = oracle.Params(eps=1.0, h=0.05, renorm_every=10 ** 6)
    S, eta = 150, 1e-6
    _, _, J, dh, de = oracle.jacobian(prm, X, P, S)

    def final(Xi, Pi, p=prm):
        st = oracle.State(Xi, Pi, p, tangent=False).advance(S)
        return np.concatenate([_unwrapped(st), st.P])

    for k in range(6):
        dz = np.zeros((6, 1)); dz[k] = eta
        plus = final(X + dz[:3], P + dz[3:])
        minus = final(X - dz[:3], P - dz[3:])
        fd = (plus - minus) / (2 * eta)
        np.testing.assert_allclose(fd.T, J[:, :, k], rtol=1e-6, atol=1e-6 * np.abs(J).max())
    # parameter directions
    for which, D in (("h", dh), ("eps", de)):
        d = 1e-7
        pp = oracle.Params(eps=prm.eps + (d if which == "eps" else 0), h=prm.h + (d if which == "h" else 0))
        pm = oracle.Params(eps=prm.eps - (d if which == "eps" else 0), h=prm.h - (d if which == "h" else 0))
        fd = (final(X, P, pp) - final(X, P, pm)) / (2 * d)
        np.testing.assert_allclose(fd.T, D, rtol=1e-5, atol=1e-5 * np.abs(D).max())
    # the run's own tangent (no renormalisation) equals J w0
    st = oracle.State(X, P, prm).advance(S)
    w0 = np.full(6, 1 / math.sqrt(6))
    np.testing.assert_allclose(st.W.T, J @ w0, rtol=1e-10, atol=1e-10 * np.abs(J).max())


def test_reversibility():
    """A symmetric composition inverts under h -> -h: S steps forward then S
    back returns the start.  Catches an asymmetric substep order."""
    X, P = _box(8, seed=9, lo=(-3.0, -3.0, -3.0), hi=(3.0, 3.0, 3.0))
    S = 400
    fw = oracle.State(X, P, oracle.Params(h=0.05), tangent=False).advance(S)
    bw = oracle.State(fw.X, fw.P, oracle.Params(h=-0.05), tangent=False).advance(S)
    X_back = bw.X + TWO_PI * (bw.lap + fw.lap)
    assert np.abs(X_back - X).max() < 1e-13 * S * 10
    assert np.abs(bw.P - P).max() < 1e-13 * S * 10


def test_renormalisation_interval_does_not_change_chi():
    """chi_t = ln(|w(t)|/|w(0)|)/t is independent of the renormalisation interval R
    (up to rounding).  Catches a lost log term or a wrong normalisation."""
    X, P = _box(16, seed=7, lo=(-3.0, -3.0, -3.0), hi=(3.0, 3.0, 3.0))
    chis = []
    for R in (1, 7, 100, 10 ** 6):
        st = oracle.State(X, P, oracle.Params(eps=1.0, h=0.05, renorm_every=R)).advance(500)
        chis.append(st.chi())
    for c in chis[1:]:
        np.testing.assert_allclose(c, chis[0], rtol=1e-11)


# ------------------------------------------------------------- potential ---
def test_potential_bound_and_derivatives():
    """Eq. 2 and the text after it: |Hp| <= 2, attained at the origin; gradient and
    Hessian agree with central differences of Hp."""
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, TWO_PI, (2000, 3))
    vals = np.array([oracle.hp(*q) for q in pts])
    assert np.abs(vals).max() <= 2.0
    assert oracle.hp(0, 0, 0) == 2.0 and oracle.hp(math.pi, 0, 0) == -2.0
    d = 1e-5
    for q in pts[:50]:
        g = oracle.grad_hp(q)
        H = oracle.hess_hp(q)
        for a in range(3):
            e = np.zeros(3); e[a] = d
            fd = (oracle.hp(*(q + e)) - oracle.hp(*(q - e))) / (2 * d)
            assert abs(fd - g[a]) < 1e-8
            fdH = (oracle.grad_hp(q + e) - oracle.grad_hp(q - e)) / (2 * d)
            np.testing.assert_allclose(fdH, H[:, a], atol=1e-8)
        assert np.allclose(H, H.T)


def test_fixed_energy_initial_conditions():
    """Sec. IV (Fig. 4 caption): p_z from the fixed-energy condition, so H(X0, P0) = E."""
    for E in (400.0, 40.0, 15.0):
        X, Pxy = inputs.grid_slice(16, E)
        P = np.zeros((3, 256)); P[:2] = Pxy
        P = oracle.pz_from_energy(E, 1.0, X, P)
        assert np.all(P[2] > 0)
        np.testing.assert_allclose(oracle.energy(1.0, X, P), E, rtol=1e-14)


# --------------------------------------------------------- paper's values ---
def test_paper_printed_values():
    """Values the paper prints (tests/golden/paper_values.json, each cited)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    from paper_1107_4107_b300 import params
    for row in g["eps_eff"]:
        assert abs(params.eps_eff(row["E"], 1.0) - row["eps_eff"]) < 1e-15
    assert g["hp_max"] == 2.0
    E = g["W_point"]["E"]
    W = np.array([math.sqrt(E), math.sqrt(E), 0.0])
    for m in g["W_point"]["resonances"]:
        assert abs(np.dot(m, W)) < 1e-12
    assert abs(np.dot(W, W) / 2 - E) < 1e-12
    assert g["realizations_step"] == 16 * 448
    assert abs(params.paper_h() - 0.01 * TWO_PI) < 1e-16


def test_chaos_sanity_paper_regimes():
    """Qualitative (Sec. IV): the triple resonance point W = (sqrt E, sqrt E, 0) is in a
    well-developed chaotic region at E = 15; a cell far from every low-order
    resonance is regular at E = 400."""
    E = 15.0
    n = 8
    X = inputs.angles(21, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3).T.copy()
    # (p_x, p_y) a little inside W so that the fixed-energy p_z is real for every angle
    P = np.zeros((3, n)); P[0] = math.sqrt(E) - 0.3; P[1] = math.sqrt(E) - 0.3
    P = oracle.pz_from_energy(E, 1.0, X, P)
    st = oracle.State(X, P, oracle.Params()).advance(100000)
    assert st.classify().mean() >= 0.75
    # far from resonances: P = (p, q, r) with |m . P| large for all low orders
    E = 400.0
    P = np.zeros((3, n)); P[0] = 9.0; P[1] = 3.0
    P = oracle.pz_from_energy(E, 1.0, X, P)
    st = oracle.State(X, P, oracle.Params()).advance(10000)
    assert st.classify().sum() == 0


# ------------------------------------------------------------- statistics ---
def test_stats_brute_force():
    """The histogram, chaotic count and moments against an independent recount."""
    rng = np.random.default_rng(3)
    chi = 10.0 ** rng.uniform(-9, 2, 5000)
    chi[:5] = [0.0, -1.0, 1e-9, 10.0, 1e-3]
    dE = rng.uniform(0, 1e-3, 5000)
    P = rng.normal(size=(3, 5000)) * [[1.0], [2.0], [3.0]]
    t = 628.3
    s = oracle.stats(chi, dE, P, t)
    lo, hi, nb = -8.0, 1.0, 200
    edges = lo + (hi - lo) * np.arange(nb + 1) / nb
    pos = chi[chi > 0]
    l10 = np.log10(pos)
    ref, _ = np.histogram(l10[(l10 >= lo) & (l10 < hi)], bins=edges)
    # values within rounding of an edge may fall either side: compare totals exactly, bins to +-1
    assert s["hist"].sum() == ref.sum()
    assert np.abs(s["hist"] - ref).max() <= 1
    assert s["under"] == np.sum(chi <= 0) + np.sum(l10 < lo)
    assert s["over"] == np.sum(l10 >= hi)
    thr = 10 * math.log(t) / t
    assert s["chaotic"] == sum(1 for c in chi if c > thr)
    assert s["dE_max"] == dE.max()
    for a in range(3):
        m = sum(P[a]) / 5000
        assert abs(s["p_mean"][a] - m) < 1e-12
        assert abs(s["p_var"][a] - sum((P[a] - m) ** 2) / 5000) < 1e-10


def test_oracle_gradient_matches_finite_differences():
    """Loss L = mean_alpha Var_i P_alpha(N): the forward-mode gradient w.r.t. (x0, p0,
    h, eps) against central differences of L (eta = 1e-6, N = 200)."""
    n = 6
    X, P = inputs.box(n, seed=0)
    prm = oracle.Params(eps=1.0, h=0.02 * math.pi)
    N = 200
    gx, gp, gh, ge, _, _ = oracle.gradient(prm, X, P, N)

    def L(Xi, Pi, p=prm):
        st = oracle.State(Xi, Pi, p, tangent=False).advance(N)
        return oracle.loss_variance(st.P)

    eta = 1e-6
    for a in range(3):
        for i in (0, 3):
            e = np.zeros((3, n)); e[a, i] = eta
            fdx = (L(X + e, P) - L(X - e, P)) / (2 * eta)
            fdp = (L(X, P + e) - L(X, P - e)) / (2 * eta)
            # relative to the gradient's scale (entries span orders of magnitude)
            assert abs(fdx - gx[a, i]) <= 1e-6 * np.abs(gx).max()
            assert abs(fdp - gp[a, i]) <= 1e-6 * np.abs(gp).max()
    d = 1e-7
    fdh = (L(X, P, oracle.Params(h=prm.h + d)) - L(X, P, oracle.Params(h=prm.h - d))) / (2 * d)
    fde = (L(X, P, oracle.Params(eps=1 + d)) - L(X, P, oracle.Params(eps=1 - d))) / (2 * d)
    assert abs(fdh - gh) <= 1e-5 * abs(gh)
    assert abs(fde - ge) <= 1e-5 * abs(ge)
