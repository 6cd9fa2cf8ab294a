"""In-kernel snapshots of the window velocity V (Sec. IV: F is built from V over
windows of Delta t): one long iterate call records the V of every window into a
caller-owned device array, identical to reading V after each window."""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def torch():
    t = pytest.importorskip("torch")
    assert t.cuda.is_available(), "GPU test needs CUDA"
    return t


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "df64", "df64f"])
def test_snapshots_equal_per_window_reads(torch, precision):
    n, W, k = 777, 50, 5
    X, P = inputs.box(n, seed=41)
    snap = torch.full((k, 3, n), float("nan"), dtype=torch.float64, device="cuda")
    a = _ens(n, precision=precision, window=W, launch_steps=37)
    a.set_state(X, P)
    a.set_snapshots(snap)
    a.iterate(k * W + 13)                 # k windows and part of the next, split over launches
    b = _ens(n, precision=precision, window=W)
    b.set_state(X, P)
    got = snap.cpu().numpy()
    for w in range(k):
        b.iterate(W)
        assert np.array_equal(got[w], b.indicator("V")), w


def test_snapshots_fp64_vs_oracle_windows(torch):
    n, W, k = 64, 40, 3
    X, P = inputs.box(n, seed=42)
    snap = torch.empty((k, 3, n), dtype=torch.float64, device="cuda")
    e = _ens(n, window=W)
    e.set_state(X, P)
    e.set_snapshots(snap)
    e.iterate(k * W)
    st = oracle.State(X, P, oracle_params(window=W))
    got = snap.cpu().numpy()
    for w in range(k):
        st.advance(W)
        assert rel_err(got[w], st.velocity()) < 1e-12, w


def test_snapshots_respect_k_max_and_clock_reset(torch):
    n, W = 100, 20
    X, P = inputs.box(n, seed=43)
    buf = torch.full((5, 3, n), float("nan"), dtype=torch.float64, device="cuda")
    e = _ens(n, window=W)
    e.set_state(X, P)
    e.set_snapshots(buf[:3])              # room for 3 of the 5 windows
    e.iterate(5 * W)
    got = buf.cpu().numpy()
    assert np.all(np.isfinite(got[:3])) and np.all(np.isnan(got[3:]))
    first = got[0].copy()
    e.set_state(inputs.box(n, seed=44)[0], P)   # clock reset: windows count from 1 again
    e.iterate(W)
    again = buf.cpu().numpy()
    assert not np.array_equal(again[0], first) and np.array_equal(again[1:3], got[1:3])
    e.set_snapshots(None)
    e.iterate(W)
    assert np.array_equal(buf.cpu().numpy()[:3], again[:3])


def test_snapshots_need_windows(torch):
    from paper_1107_4107_b300.api import ArnoldError
    snap = torch.empty((2, 3, 10), dtype=torch.float64, device="cuda")
    e = _ens(10)                          # window = 0: no windows to record
    with pytest.raises(ArnoldError):
        e.set_snapshots(snap)
