"""DF64F path (double-float state, products, sums and tangent, with sines and
cosines to ~3e-10) against the FP64 oracle.

Bars, derived from the sincos error.  The reduced argument r = x - theta_j is
formed in FP32 with three roundings at |r| <= D/2 ~ 1.5e-3 (half an ulp there
is 5.8e-11), the small terms C r + S cm add one more, and the neglected
C_lo r and r^4/24 stay below 5e-11: |sin - sin_exact|, |cos - cos_exact| <=
3e-10 (measured 2.3e-10).  Everything else is double-float, so the trajectory
error is that sincos error times the kick size, as in the compensated-FP32
mode whose 9e-8 sincos gives its 3e-8 / 3e-7 / 3e-6 bars (1 / 100 / 1000
steps); scaled by 3e-10 / 9e-8: 1e-10 after one step, 1e-9 after 100 (all
cells), 1e-8 after 1000 (every cell, times its own tangent growth), on
displacement, momenta, V and the FTLE.  The tangent components depend on second derivatives of the flow,
which grow like t^2 (the FP64 test's argument): 1e-9 x (100 h)^2 = 4e-8 at
100 steps.  Grid inputs hold cells near resonances, where the bound is scaled
by each cell's own tangent growth exp(chi t).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_grid_state, oracle_params, rel_err

pytestmark = pytest.mark.gpu
SINCOS_BAR = 3e-10
BOUNDS = {1: 1e-10, 10: 1e-9, 100: 1e-9}
LONG_BAR = 1e-8
TANGENT_BAR_100 = 1e-9 * (100 * 0.02 * math.pi) ** 2


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, precision="df64f", **kw)


def test_df64f_sincos_accuracy():
    import torch
    x0 = np.linspace(0.0, 2 * math.pi, 400001)
    hi = x0.astype(np.float32)
    lo = (x0 - hi.astype(np.float64)).astype(np.float32)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    xd = torch.tensor(x, device="cuda")
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    e = _ens(8)
    e.debug_sincos(xd, s, c, "df64f")
    es = np.abs(s.cpu().numpy() - np.sin(x)).max()
    ec = np.abs(c.cpu().numpy() - np.cos(x)).max()
    assert es < SINCOS_BAR and ec < SINCOS_BAR, (es, ec)


@pytest.mark.parametrize("n", [33, 1000])
def test_df64f_state_parity_all_cells(n):
    X, P = inputs.box(n, seed=41)
    st = oracle.State(X, P, oracle_params(R=10))
    e = _ens(n, renorm_every=10)
    e.set_state(X, P)
    for S in (1, 9, 90):
        e.iterate(S)
        st.advance(S)
        bar = BOUNDS[st.steps]
        assert rel_err(e.indicator("dX"), st.unwrapped_displacement()) < bar
        assert rel_err(e.indicator("P"), st.P) < bar
    assert rel_err(e.indicator("V"), st.velocity()) < BOUNDS[100]
    assert rel_err(e.indicator("chi"), st.chi()) < BOUNDS[100]
    assert rel_err(e.indicator("tangent"), st.W) < TANGENT_BAR_100


def test_df64f_long_horizon_growth_scaled():
    """1000 steps, every cell: ten times the 100-step bar (the sincos errors add up
    over ten times the steps), times the cell's own growth G = exp(chi t)."""
    from parity import cell_growth, growth_scaled
    n = 1024
    X, P = inputs.box(n, seed=42)
    st = oracle.State(X, P, oracle_params()).advance(1000, threads=4)
    e = _ens(n)
    e.set_state(X, P)
    e.iterate(1000)
    g = cell_growth(st)
    report = {}
    for kind, ref in (("dX", st.unwrapped_displacement()), ("P", st.P), ("chi", st.chi())):
        ok, worst = growth_scaled(e.indicator(kind), ref, g, LONG_BAR)
        report[kind] = worst
        assert ok, (kind, worst)
    print("df64f worst err / bar:", report)


def _growth_scaled(got, ref, st, bound):
    """Per cell: the bound times the cell's own tangent growth exp(chi t) (first-order
    error propagation; grids hold cells near resonances that stretch errors within
    100 steps, as the compensated-FP32 full-size test states)."""
    from parity import cell_growth, growth_scaled
    return growth_scaled(got, ref, cell_growth(st), bound)


@pytest.mark.parametrize("E", [400.0, 40.0, 15.0])
def test_df64f_grid_parity(E):
    G = 32
    st = oracle_grid_state(G, E, oracle_params())
    e = _ens(G * G)
    e.init_grid(G, E)
    e.iterate(100)
    st.advance(100, threads=4)
    for got, ref in ((e.indicator("dX"), st.unwrapped_displacement()), (e.indicator("P"), st.P)):
        ok, worst = _growth_scaled(got, ref, st, BOUNDS[100])
        assert ok, worst


def test_df64f_sincos_accuracy_large_angles():
    """Angles up to 12 + h |q| < 172 rad within a step keep the 3e-10 bound."""
    import torch
    x0 = np.linspace(-172.0, 172.0, 400001)
    hi = x0.astype(np.float32)
    lo = (x0 - hi.astype(np.float64)).astype(np.float32)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    xd = torch.tensor(x, device="cuda")
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    e = _ens(8)
    e.debug_sincos(xd, s, c, "df64f")
    es = np.abs(s.cpu().numpy() - np.sin(x)).max()
    ec = np.abs(c.cpu().numpy() - np.cos(x)).max()
    assert es < SINCOS_BAR and ec < SINCOS_BAR, (es, ec)


def test_df64f_large_step_angle_parity():
    """h |q| ~ 100 rad per step (the batched scan's high-energy sets) against the
    oracle, with the 1 / 10-step bars (the kick here, 2 w h eps ~ 0.4, is of the
    size of the grid tests')."""
    n = 200
    X, P = inputs.box(n, seed=43, lo=(300.0, 200.0, 100.0), hi=(301.0, 201.0, 101.0))
    h = 0.2
    st = oracle.State(X, P, oracle_params(h=h, R=5))
    e = _ens(n, h=h, renorm_every=5)
    e.set_state(X, P)
    for S, bar in ((1, BOUNDS[1]), (9, BOUNDS[10])):
        e.iterate(S)
        st.advance(S)
        assert rel_err(e.indicator("dX"), st.unwrapped_displacement()) < bar
        assert rel_err(e.indicator("P"), st.P) < bar
    e.sync()


def test_df64f_range_resume_and_no_adjoint():
    from paper_1107_4107_b300._lib import ArnoldError, ERANGE, EUNSUPPORTED
    X, P = inputs.box(64, seed=1, lo=(1000.0, 1000.0, 1000.0), hi=(1001.0, 1001.0, 1001.0))
    e = _ens(64, h=0.1, renorm_every=1)
    e.set_state(X, P)
    e.iterate(2)
    with pytest.raises(ArnoldError) as ex:
        e.sync()
    assert ex.value.status == ERANGE
    X, P = inputs.box(500, seed=5)
    ref = _ens(500, renorm_every=7)
    ref.set_state(X, P)
    ref.iterate(120)
    a = _ens(500, renorm_every=7)
    a.set_state(X, P)
    a.iterate(50)
    b = _ens(500, renorm_every=7)
    b.restore(a.checkpoint())
    b.iterate(70)
    for k in ("dX", "P", "tangent", "chi"):
        assert np.array_equal(ref.indicator(k), b.indicator(k)), k
    with pytest.raises(ArnoldError) as ex:
        b.forward_ckpt(10)
    assert ex.value.status == EUNSUPPORTED


def test_df64f_full_size_grid_sampled_cells():
    """The 2048 x 2048 scan (default launch configuration): 256 sampled cells
    against the FP64 oracle one by one, 100 steps."""
    G, E = 2048, 400.0
    e = _ens(G * G)
    e.init_grid(G, E)
    e.iterate(100)
    cells = inputs.sample_cells(G * G, 256, seed=5)
    st = oracle_grid_state(G, E, oracle_params(), cells=cells).advance(100, threads=4)
    for got, ref in ((e.indicator("dX")[:, cells], st.unwrapped_displacement()), (e.indicator("P")[:, cells], st.P)):
        ok, worst = _growth_scaled(got, ref, st, BOUNDS[100])
        assert ok, worst
    assert rel_err(e.indicator("chi")[cells], st.chi()) < BOUNDS[100]
    assert rel_err(e.indicator("tangent")[:, cells], st.W) < TANGENT_BAR_100
