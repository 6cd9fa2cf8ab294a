"""DF64 path (double-float state and kicks on the FP32 pipes) against the FP64
oracle at the FP64 tolerance.

A double-float word carries ~48 significant bits against FP64's 53, so every
rounding (and the initial conversion of the state) is ~2^5 = 32 times coarser
than in the FP64 kernel; the trajectory (displacement, momenta, V) is held to
the FP64 bound scaled by that factor, 3e-11 relative (measured ~2e-12 over
1000 steps).  The tangent vector is double-float too, so it and the FTLE are
held to the FP64 kernel's bars scaled the same way: 3e-11 on all cells to 100
steps, and to 1000 steps on every cell 32 x 1e-12 times the cell's own
tangent growth G = exp(chi t) (G^2 for the tangent components, whose
second-derivative growth the FP64 test derives).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_grid_state, oracle_params, rel_err

pytestmark = pytest.mark.gpu
TOL = 3e-11


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, precision="df64", **kw)


def test_df64_sincos_accuracy():
    import torch
    # inputs exactly representable as float pairs (hi + lo), so the test sees the
    # sincos error and not the 48-bit rounding of the argument
    x0 = np.linspace(0.0, 2 * math.pi, 400001)
    hi = x0.astype(np.float32)
    lo = (x0 - hi.astype(np.float64)).astype(np.float32)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    xd = torch.tensor(x, device="cuda")
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    e = _ens(8)
    e.debug_sincos(xd, s, c, "df64")
    es = np.abs(s.cpu().numpy() - np.sin(x)).max()
    ec = np.abs(c.cpu().numpy() - np.cos(x)).max()
    # a float pair resolves ~2^-48 relative: a few of its last places ~ 1e-14
    assert es < 2e-14 and ec < 2e-14, (es, ec)


@pytest.mark.parametrize("n", [33, 1000])
def test_df64_state_parity_all_cells(n):
    X, P = inputs.box(n, seed=41)
    st = oracle.State(X, P, oracle_params(R=10))
    e = _ens(n, renorm_every=10)
    e.set_state(X, P)
    for S in (1, 9, 90):
        e.iterate(S)
        st.advance(S)
        assert rel_err(e.indicator("dX"), st.unwrapped_displacement()) < TOL
        assert rel_err(e.indicator("P"), st.P) < TOL
    assert rel_err(e.indicator("V"), st.velocity()) < TOL
    assert rel_err(e.indicator("tangent"), st.W) < TOL
    assert rel_err(e.indicator("chi"), st.chi()) < TOL
    assert np.max(np.abs(e.indicator("dE_max") - st.dE_max)) < 1e-9


def test_df64_long_horizon_growth_scaled():
    """1000 steps, every cell: the FP64 kernel's growth-scaled bars (1e-12 G on
    state and FTLE, 1e-12 G^2 on the tangent, G = exp(chi t) from the oracle)
    times 2^5 for the double-float word."""
    from parity import cell_growth, growth_scaled
    n = 1024
    X, P = inputs.box(n, seed=42)
    st = oracle.State(X, P, oracle_params()).advance(1000, threads=4)
    e = _ens(n)
    e.set_state(X, P)
    e.iterate(1000)
    g = cell_growth(st)
    report = {}
    for kind, ref, power in (("dX", st.unwrapped_displacement(), 1), ("P", st.P, 1), ("chi", st.chi(), 1),
                             ("tangent", st.W, 2)):
        ok, worst = growth_scaled(e.indicator(kind), ref, g, 32 * 1e-12, power)
        report[kind] = worst
        assert ok, (kind, worst)
    print("df64 worst err / bar:", report)


@pytest.mark.parametrize("E", [400.0, 40.0, 15.0])
def test_df64_grid_parity(E):
    G = 32
    st = oracle_grid_state(G, E, oracle_params())
    e = _ens(G * G)
    e.init_grid(G, E)
    e.iterate(100)
    st.advance(100, threads=4)
    assert rel_err(e.indicator("dX"), st.unwrapped_displacement()) < TOL
    assert rel_err(e.indicator("P"), st.P) < TOL


def test_df64_sincos_accuracy_large_angles():
    """Within a step an angle reaches 12 + h |q| < 172 rad before it is reduced:
    the sincos of such pairs keeps its accuracy (x.hi - j d1 stays exact)."""
    import torch
    x0 = np.linspace(-172.0, 172.0, 400001)
    hi = x0.astype(np.float32)
    lo = (x0 - hi.astype(np.float64)).astype(np.float32)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    xd = torch.tensor(x, device="cuda")
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    e = _ens(8)
    e.debug_sincos(xd, s, c, "df64")
    es = np.abs(s.cpu().numpy() - np.sin(x)).max()
    ec = np.abs(c.cpu().numpy() - np.cos(x)).max()
    assert es < 2e-14 and ec < 2e-14, (es, ec)


def test_df64_large_step_angle_parity():
    """Fast trajectories (h |q| ~ 100 rad per step, as in the batched scan's
    high-energy sets) against the oracle: angles run far past the 12 rad
    reduction point within every step and must be followed exactly."""
    n = 200
    X, P = inputs.box(n, seed=43, lo=(300.0, 200.0, 100.0), hi=(301.0, 201.0, 101.0))
    h = 0.2   # h |q_u| = h |p_x + p_y| ~ 100
    st = oracle.State(X, P, oracle_params(h=h, R=5))
    e = _ens(n, h=h, renorm_every=5)
    e.set_state(X, P)
    for S in (1, 4, 15):
        e.iterate(S)
        st.advance(S)
        assert rel_err(e.indicator("dX"), st.unwrapped_displacement()) < TOL
        assert rel_err(e.indicator("P"), st.P) < TOL
        assert rel_err(e.indicator("chi"), st.chi()) < TOL
    e.sync()


def test_df64_range_is_reported():
    """h |q| beyond the mode's range (160 rad per step) is reported as ERANGE, not
    computed wrong."""
    from paper_1107_4107_b300._lib import ArnoldError, ERANGE
    X, P = inputs.box(64, seed=1, lo=(1000.0, 1000.0, 1000.0), hi=(1001.0, 1001.0, 1001.0))
    e = _ens(64, h=0.1, renorm_every=1)
    e.set_state(X, P)
    e.iterate(2)
    with pytest.raises(ArnoldError) as ex:
        e.sync()
    assert ex.value.status == ERANGE


def test_df64_resume_bitwise_and_no_adjoint():
    from paper_1107_4107_b300._lib import ArnoldError, EUNSUPPORTED
    X, P = inputs.box(500, seed=5)
    ref = _ens(500, renorm_every=7)
    ref.set_state(X, P)
    ref.iterate(120)
    a = _ens(500, renorm_every=7)
    a.set_state(X, P)
    a.iterate(50)
    blob = a.checkpoint()
    b = _ens(500, renorm_every=7)
    b.restore(blob)
    b.iterate(70)
    for k in ("dX", "P", "tangent", "chi"):
        assert np.array_equal(ref.indicator(k), b.indicator(k)), k
    with pytest.raises(ArnoldError) as ex:
        b.forward_ckpt(10)
    assert ex.value.status == EUNSUPPORTED


def test_df64_full_size_grid_sampled_cells():
    """The 2048 x 2048 scan in double-float (default launch configuration): 256 sampled
    cells against the FP64 oracle one by one, 100 steps (state, tangent, FTLE)."""
    G, E = 2048, 400.0
    e = _ens(G * G)
    e.init_grid(G, E)
    e.iterate(100)
    cells = inputs.sample_cells(G * G, 256, seed=5)
    st = oracle_grid_state(G, E, oracle_params(), cells=cells).advance(100, threads=4)
    assert rel_err(e.indicator("dX")[:, cells], st.unwrapped_displacement()) < TOL
    assert rel_err(e.indicator("P")[:, cells], st.P) < TOL
    assert rel_err(e.indicator("tangent")[:, cells], st.W) < TOL
    assert rel_err(e.indicator("chi")[cells], st.chi()) < TOL
