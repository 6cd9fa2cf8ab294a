"""Pins of the oracle's sphere ensembles, area tracking and V histogram (Sec. IV),
and of the seeded sphere / Gaussian generators."""
import math

import numpy as np

import oracle
from paper_1107_4107_b300 import inputs

TWO_PI = 2 * math.pi


def test_sphere_generator_is_uniform():
    X, nh = inputs.sphere_directions(200000, seed=4)
    np.testing.assert_allclose(np.sum(nh * nh, axis=0), 1.0, atol=1e-14)
    c, _ = np.histogram(nh[2], bins=20, range=(-1, 1))
    assert np.abs(c / 10000.0 - 1).max() < 0.05                  # cos theta uniform (Archimedes)
    phi = np.mod(np.arctan2(nh[1], nh[0]), TWO_PI)
    c, _ = np.histogram(phi, bins=20, range=(0, TWO_PI))
    assert np.abs(c / 10000.0 - 1).max() < 0.05
    assert X.min() >= 0 and X.max() < TWO_PI
    _, nh2 = inputs.sphere_directions(1000, seed=4, cos_range=(0.1, 0.2), phi_range=(1.0, 1.3))
    assert nh2[2].min() >= 0.1 and nh2[2].max() <= 0.2


def test_gaussian_generator_moments():
    _, Pxy = inputs.gaussian_velocities(400000, center=(3.0, -2.0), sigma=0.01, seed=2)
    assert abs(Pxy[0].mean() - 3.0) < 1e-4 and abs(Pxy[1].mean() + 2.0) < 1e-4
    assert abs(Pxy[0].std() / 0.01 - 1) < 0.01 and abs(Pxy[1].std() / 0.01 - 1) < 0.01


def test_momenta_on_shell_have_the_energy():
    X, nh = inputs.sphere_directions(500, seed=1)
    for E in (400.0, 15.0):
        P = oracle.momenta_on_shell(E, 1.0, X, nh)
        np.testing.assert_allclose(oracle.energy(1.0, X, P), E, rtol=1e-14)
        np.testing.assert_allclose(P / np.sqrt(np.sum(P * P, axis=0)), nh, atol=1e-14)


def test_tracking_closed_form_at_zero_coupling():
    """eps = 0: momenta never change, so a trajectory leaves the patch at the first
    sample iff it starts outside."""
    X, nh = inputs.sphere_directions(300, seed=5)
    P = 20.0 * nh
    patch = (-0.3, 0.5, 0.5, 2.5)
    c = nh[2]
    phi = np.mod(np.arctan2(nh[1], nh[0]), TWO_PI)
    outside = ~((c >= patch[0]) & (c <= patch[1]) & (phi >= patch[2]) & (phi <= patch[3]))
    _, PN, left = oracle.track_patch(oracle.Params(eps=0.0, renorm_every=10), X, P, 50, patch)
    assert np.array_equal(PN, P)
    assert np.array_equal(left.astype(bool), outside)


def test_velocity_histogram_closed_form_at_zero_coupling():
    """eps = 0: V = P0, so F is the histogram of the initial directions."""
    X, nh = inputs.sphere_directions(5000, seed=6)
    P = 10.0 * nh
    st = oracle.State(X, P, oracle.Params(eps=0.0), tangent=False).advance(40)
    H = oracle.velocity_histogram(st.velocity(), 16, 32)
    c = nh[2]
    phi = np.mod(np.arctan2(nh[1], nh[0]), TWO_PI)
    ref, _, _ = np.histogram2d(c, phi, bins=[16, 32], range=[[-1, 1], [0, TWO_PI]])
    assert H.sum() == 5000
    assert np.abs(H - ref).sum() <= 4        # only values on a cell edge may move
    keep = np.zeros(5000, dtype=np.uint8)
    keep[::2] = 1
    assert oracle.velocity_histogram(st.velocity(), 16, 32, keep=keep).sum() == 2500
