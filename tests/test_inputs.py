"""The seeded input generator shared by both sides (no method arithmetic)."""
import json
import math
import os

import numpy as np

from paper_1107_4107_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    got = inputs.splitmix64(g["seed"], np.arange(5, dtype=np.uint64))
    assert [f"{int(v):016x}" for v in got] == g["outputs_hex"]


def test_angles_in_range_and_uniform():
    a = inputs.angles(0, np.arange(200000, dtype=np.uint64))
    assert a.min() >= 0.0 and a.max() < 2 * math.pi
    hist, _ = np.histogram(a, bins=20, range=(0, 2 * math.pi))
    assert np.abs(hist / 10000.0 - 1).max() < 0.05


def test_grid_slice_layout_and_shards():
    G = 16
    X, Pxy = inputs.grid_slice(G, 400.0)
    a = inputs.grid_halfwidth(400.0, 1.0)
    assert X.shape == (3, G * G) and Pxy.shape == (2, G * G)
    # row-major: t = j * G + i, p_x from i, p_y from j
    assert np.allclose(Pxy[0, :G], -a + 2 * a * (np.arange(G) + 0.5) / G)
    assert np.all(Pxy[1, :G] == Pxy[1, 0])
    assert np.all(np.abs(Pxy) < a)
    # a band of rows is exactly the slice of the full grid
    Xs, Ps = inputs.grid_slice(G, 400.0, rows=(5, 9))
    assert np.array_equal(Xs, X[:, 5 * G:9 * G]) and np.array_equal(Ps, Pxy[:, 5 * G:9 * G])


def test_box_ranges_and_offset():
    X, P = inputs.box(1000, seed=0)
    assert np.all((P[0] >= 10) & (P[0] < 11)) and np.all((P[2] >= 25) & (P[2] < 26))
    X2, P2 = inputs.box(10, seed=0, offset=990)
    assert np.array_equal(X2, X[:, 990:]) and np.array_equal(P2, P[:, 990:])


def test_sample_cells_distinct_sorted():
    c = inputs.sample_cells(2048 * 2048, 4096)
    assert len(c) == 4096 and len(np.unique(c)) == 4096 and np.all(np.diff(c) > 0)
