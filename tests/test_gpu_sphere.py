"""Sphere ensembles, area tracking and the density of V on the momentum sphere
(Sec. IV, Figs. 2-4) on the GPU against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import rel_err

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


def test_shell_initial_conditions():
    n = 4096
    X, nh = inputs.sphere_directions(n, seed=3)
    e = _ens(n)
    e.init_sphere(400.0, seed=3)
    assert rel_err(e.indicator("P"), oracle.momenta_on_shell(400.0, 1.0, X, nh)) < 1e-14
    X2, Pxy = inputs.gaussian_velocities(n, center=(math.sqrt(15.0) - 0.3, math.sqrt(15.0) - 0.3), sigma=0.01, seed=4)
    e.init_gaussian(15.0, center=(math.sqrt(15.0) - 0.3, math.sqrt(15.0) - 0.3), sigma=0.01, seed=4)
    P = np.zeros((3, n)); P[:2] = Pxy
    assert rel_err(e.indicator("P"), oracle.pz_from_energy(15.0, 1.0, X2, P)) < 1e-14
    assert np.max(e.indicator("dE")) < 1e-12 * 400


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_area_tracking_matches_oracle(precision):
    """A patch of the sphere at E = 15 (moderate perturbation, Fig. 3): trajectories
    flagged for leaving the patch at any sample every R = 10 steps."""
    n, S, E = 3000, 300, 15.0
    patch = (0.2, 0.45, 0.6, 1.1)
    X, nh = inputs.sphere_directions(n, seed=8, cos_range=patch[:2], phi_range=patch[2:])
    P = oracle.momenta_on_shell(E, 1.0, X, nh)
    _, _, left = oracle.track_patch(oracle.Params(renorm_every=10), X, P, S, patch)
    e = _ens(n, precision=precision, renorm_every=10)
    e.init_sphere(E, seed=8, cos_range=patch[:2], phi_range=patch[2:])
    e.track_patch(*patch)
    e.iterate(S)
    got = e.indicator("left")
    assert 0.02 < left.mean() < 0.98
    # FP64: identical up to decisions within rounding of the patch edge;
    # FP32C: trajectories differ at ~1e-7, so a few edge crossings may differ
    allowed = 3 if precision == "fp64" else max(10, n // 100)
    assert int(np.sum(got != left)) <= allowed


def test_velocity_histogram_matches_oracle():
    n, S, E = 20000, 200, 400.0
    X, nh = inputs.sphere_directions(n, seed=9)
    st = oracle.State(X, oracle.momenta_on_shell(E, 1.0, X, nh), oracle.Params(), tangent=False)
    st.advance(S, threads=8)
    ref = oracle.velocity_histogram(st.velocity(), 24, 48)
    e = _ens(n, tangent=False)
    e.init_sphere(E, seed=9)
    e.iterate(S)
    got = e.velocity_histogram(24, 48)
    assert got.sum() == ref.sum() == n
    assert np.abs(got.astype(np.int64) - ref).sum() <= 4
    # accumulation over two calls (time-averaged F) and the device path
    got2 = e.velocity_histogram(24, 48, out=got.copy(), accumulate=True)
    assert np.array_equal(got2, 2 * got)


def test_filtered_histogram_counts_only_tracked_trajectories():
    n, E = 5000, 15.0
    patch = (0.2, 0.45, 0.6, 1.1)
    e = _ens(n, tangent=False, renorm_every=5)
    e.init_sphere(E, seed=10, cos_range=patch[:2], phi_range=patch[2:])
    e.track_patch(*patch)
    e.iterate(200)
    left = e.indicator("left")
    H = e.velocity_histogram(10, 10, patch=patch, filtered=True)
    V = e.indicator("V")
    c = V[2] / np.sqrt(np.sum(V * V, axis=0))
    phi = np.mod(np.arctan2(V[1], V[0]), TWO_PI)
    inside = (c >= patch[0]) & (c <= patch[1]) & (phi >= patch[2]) & (phi <= patch[3])
    assert H.sum() == int(np.sum(inside & (left == 0)))


@pytest.mark.parametrize("precision", ["fp64", "df64f"])
def test_tracked_run_resumes_bitwise_from_checkpoint(precision):
    """A checkpoint taken with area tracking on carries the flags: a fresh
    context tracking the same patch, restored and continued, ends with the
    uninterrupted run's flags, state and filtered F; a context that does not
    track (or tracks another patch) is refused."""
    from paper_1107_4107_b300._lib import ArnoldError, EINVAL
    n, E = 4000, 15.0
    patch = (0.2, 0.45, 0.6, 1.1)

    def fresh():
        e = _ens(n, tangent=False, renorm_every=5, precision=precision)
        e.init_sphere(E, seed=12, cos_range=patch[:2], phi_range=patch[2:])
        e.track_patch(*patch)
        return e

    ref = fresh()
    ref.iterate(300)
    a = fresh()
    a.iterate(120)
    blob = a.checkpoint()
    assert 0 < int(a.indicator("left").sum()) < n    # some flags are set when the checkpoint is taken
    b = _ens(n, tangent=False, renorm_every=5, precision=precision)
    b.track_patch(*patch)
    b.restore(blob)
    b.iterate(180)
    assert np.array_equal(b.indicator("left"), ref.indicator("left"))
    assert np.array_equal(b.indicator("P"), ref.indicator("P"))
    assert np.array_equal(b.velocity_histogram(10, 10, patch=patch, filtered=True),
                          ref.velocity_histogram(10, 10, patch=patch, filtered=True))
    for other in (None, (0.2, 0.45, 0.6, 1.2)):
        c = _ens(n, tangent=False, renorm_every=5, precision=precision)
        if other:
            c.track_patch(*other)
        with pytest.raises(ArnoldError) as ex:
            c.restore(blob)
        assert ex.value.status == EINVAL


@pytest.mark.parametrize("precision", ["fp64", "df64f"])
def test_device_sphere_draws_match_the_generator(precision):
    """arnold_init_sphere draws the host generator's counters on the device: angles
    equal, momenta on the energy shell along the generator's directions (CUDA sin/cos
    of phi against libm: ~1e-16), for a patch and an offset into the stream."""
    from parity import angle_dist
    n, E, off = 5000, 400.0, 123457
    patch = (-0.3, 0.8, 0.5, 4.0)
    X, nh = inputs.sphere_directions(n, seed=21, cos_range=patch[:2], phi_range=patch[2:], offset=off)
    e = _ens(n, precision=precision)
    e.init_sphere(E, seed=21, cos_range=patch[:2], phi_range=patch[2:], offset=off)
    tol = 1e-14 if precision == "fp64" else 1e-13
    assert np.max(angle_dist(e.indicator("X"), X)) < tol
    assert rel_err(e.indicator("P"), oracle.momenta_on_shell(E, 1.0, X, nh)) < tol
    assert np.max(e.indicator("dE")) < 1e-12 * E
    e.sync()


def test_device_gaussian_keeps_exactly_the_draws_with_a_real_pz():
    """arnold_init_gaussian at W = (sqrt E, sqrt E, 0), E = 15 (Fig. 4), where the
    energy condition rejects many draws: the ensemble holds the first n draws that
    the oracle's own energy condition accepts, in order, and reports how many draws
    it examined; an offset continues the stream; a cloud off the shell is ERANGE."""
    from paper_1107_4107_b300._lib import ArnoldError, ERANGE
    from parity import angle_dist
    n, E, sigma = 3000, 15.0, 0.01
    W = math.sqrt(E)
    for off in (0, 77777):
        cand = 4 * n
        X, Pxy = inputs.gaussian_velocities(cand, (W, W), sigma, seed=5, offset=off)
        P = np.zeros((3, cand))
        P[:2] = Pxy
        Po = oracle.pz_from_energy(E, 1.0, X, P)
        ok = np.isfinite(Po[2])
        assert 0.05 < ok.mean() < 0.95 and ok.sum() >= n
        e = _ens(n, tangent=False)
        drawn = e.init_gaussian(E, (W, W), sigma, seed=5, offset=off)
        assert drawn == int(np.nonzero(ok)[0][n - 1]) + 1
        assert np.max(angle_dist(e.indicator("X"), X[:, ok][:, :n])) < 1e-14
        assert rel_err(e.indicator("P"), Po[:, ok][:, :n]) < 1e-13
        e.sync()
    e = _ens(64, tangent=False)
    with pytest.raises(ArnoldError) as ex:
        e.init_gaussian(E, (10.0, 10.0), sigma, seed=5)
    assert ex.value.status == ERANGE
