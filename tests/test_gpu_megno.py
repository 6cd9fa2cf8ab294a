"""MEGNO on the GPU (FP64, FP32C, DF64) vs the oracle, element by element on the
same seeded inputs, plus the free-flow closed form and bitwise invariances.

Bars.  MEGNO is a weighted sum of the renormalisation logs; by summation by
parts Y_m = 2 L_m - (2/m) sum_{k<m} L_k (L_k the log sum after k
renormalisations), so |dY| <= 4 max_k |dL_k| and |d<Y>| likewise.  FP64: the
log sums agree to rounding (the FTLE bar, 1e-12 relative) over 100 steps on
all cells; to 1000 steps every cell's tangent is held to 1e-12 G^2 (G its own
tangent growth exp(chi t)), so MEGNO to 4e-12 G^2.  FP32C carries the tangent in FP32, whose log-sum error grows
about linearly in the step count (bar below); DF64 carries it in double-float
(~48 bits), held to the FP64 bars x 2^5.  The tests check the
summation-by-parts bound itself against both sides' recorded log-sum
histories.  DF64F (double-float with a ~3e-10 sincos) holds its log sums to
its 1000-step FTLE bar times t.  The eps = 0 closed form has no Hessian, so
there FP32C is held to 4e-6 t and DF64 and DF64F to 32 x 1e-12.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, megno=True, **kw)


def _megno_err(ens, st, mask=None):
    sel = (lambda a: a[mask]) if mask is not None else (lambda a: a)
    return max(rel_err(sel(ens.indicator("megno")), sel(st.megno_mean())),
               rel_err(sel(ens.indicator("megno_y")), sel(st.megno_y())))


@pytest.mark.parametrize("n", [1, 33, 1000])
def test_megno_fp64_all_cells(n):
    X, P = inputs.box(n, seed=21)
    prm = oracle_params(R=10)
    st = oracle.State(X, P, prm)
    ens = _ens(n, renorm_every=10)
    ens.set_state(X, P)
    for S in (1, 9, 90):
        ens.iterate(S)
        st.advance(S)
        assert rel_err(ens.indicator("logsum"), st.logsum) < 1e-12
        assert _megno_err(ens, st) < 1e-12, (st.steps, _megno_err(ens, st))


def test_megno_fp64_long_growth_scaled():
    """1000 steps, every cell: 4 x the FP64 tangent bar 1e-12 G^2 (G = exp(chi t)
    from the oracle), by the summation-by-parts bound."""
    from parity import cell_growth, growth_scaled
    X, P = inputs.box(512, lo=(-4.0, -4.0, 20.0), hi=(4.0, 4.0, 21.0), seed=22)
    prm = oracle_params(R=10)
    st = oracle.State(X, P, prm).advance(1000, threads=4)
    ens = _ens(512, renorm_every=10)
    ens.set_state(X, P)
    ens.iterate(1000)
    g = cell_growth(st)
    for kind, ref in (("megno", st.megno_mean()), ("megno_y", st.megno_y())):
        ok, worst = growth_scaled(ens.indicator(kind), ref, g, 4e-12, 2)
        assert ok, (kind, worst)


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "df64", "df64f"])
def test_megno_free_flow_closed_form(precision):
    """eps = 0: |w(t)|^2 = ((1 + t)^2 + 1) / 2 for w0 = (1, ..., 1)/sqrt 6 (Sec. II
    free rotation), independent of the oracle."""
    R, m = 7, 40
    X, P = inputs.box(64, seed=23)
    ens = _ens(64, eps=0.0, renorm_every=R, precision=precision)
    ens.set_state(X, P)
    ens.iterate(R * m + 3)
    h = 0.02 * math.pi
    t = R * h * np.arange(m + 1)
    lnN = 0.5 * np.log(((1.0 + t) ** 2 + 1.0) / 2.0)
    j = np.arange(1, m + 1)
    Y = 2.0 * np.cumsum(j * np.diff(lnN)) / j
    tol = {"fp64": 1e-12, "df64": 32e-12, "df64f": 32e-12, "fp32c": 4e-6 * (R * m * h)}[precision]
    assert rel_err(ens.indicator("megno_y"), np.full(64, Y[-1])) < tol
    assert rel_err(ens.indicator("megno"), np.full(64, Y.mean())) < tol


# FP32 tangent: ~15 rounded operations per step (2^-24 each) perturb w, and the flow
# shears what was injected at step s for the remaining steps, so the relative error
# of |w| -- the log-sum error -- grows about linearly with the step count N:
# |dL| <= 2 * 15 * 2^-24 * N.
LOG_BAR_PER_STEP = 2.0 * 15.0 * 2.0 ** -24


@pytest.mark.parametrize("precision", ["fp32c", "df64", "df64f"])
@pytest.mark.parametrize("n", [33, 700])
def test_megno_pair_modes_vs_oracle(precision, n):
    """Ragged sizes (padding slots repeat the last trajectory and must not add to its
    sums a second time); every cell over 1000 steps.  Both sides' log sums are
    read after every renormalisation, so the summation-by-parts bound
    |dY|, |d<Y>| <= 4 max_k |dL_k| is checked exactly, and the log sums against the
    FP32-tangent bar above (FP32C), the FP64 tangent bar 1e-12 G^2 x 2^5 (DF64) or
    the DF64F FTLE bar times t, each times the cell's own tangent growth G."""
    X, P = inputs.box(n, lo=(-4.0, -4.0, 20.0), hi=(4.0, 4.0, 21.0), seed=24)
    R, m = 20, 50
    st = oracle.State(X, P, oracle_params(R=R))
    ens = _ens(n, renorm_every=R, precision=precision)
    ens.set_state(X, P)
    dL = np.zeros(n)
    for _ in range(m):
        st.advance(R, threads=4)
        ens.iterate(R)
        dL = np.maximum(dL, np.abs(ens.indicator("logsum") - st.logsum))
    from parity import cell_growth
    g = cell_growth(st)
    for kind, ref in (("megno", st.megno_mean()), ("megno_y", st.megno_y())):
        d = np.abs(ens.indicator(kind) - ref)
        assert np.all(d <= 4.0 * dL + 1e-12 * (1.0 + np.abs(ref))), kind
    # per cell, times its own tangent growth G: FP32C the FP32-tangent bar; DF64 the
    # FP64 tangent bar 1e-12 G^2 x 2^5; DF64F its 1000-step FTLE bar times t
    bar = {"fp32c": LOG_BAR_PER_STEP * R * m * g, "df64": 32 * 1e-12 * g ** 2,
           "df64f": 1e-8 * R * m * 0.02 * math.pi * g}[precision]
    worst = float(np.max(dL / bar))
    print(f"{precision} n={n}: max |d log sum| / bar = {worst:.2e}")
    assert worst < 1.0, worst
    # the last trajectory (the one padding slots repeat) holds the same bound
    ref_last = st.megno_mean()[-1]
    assert abs(ens.indicator("megno")[-1] - ref_last) <= 4.0 * dL[-1] + 1e-12 * (1.0 + abs(ref_last))


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "df64", "df64f"])
def test_megno_launch_split_and_resume_bitwise(precision):
    X, P = inputs.box(300, seed=25)
    ref = _ens(300, renorm_every=10, precision=precision)
    ref.set_state(X, P)
    ref.iterate(500)
    split = _ens(300, renorm_every=10, precision=precision, launch_steps=37)
    split.set_state(X, P)
    split.iterate(123)
    blob = split.checkpoint()
    other = _ens(300, renorm_every=10, precision=precision)
    other.restore(blob)
    other.iterate(377)
    split.iterate(377)
    for k in ("megno", "megno_y", "logsum"):
        assert np.array_equal(ref.indicator(k), split.indicator(k)), k
        assert np.array_equal(ref.indicator(k), other.indicator(k)), k


def test_megno_off_and_mismatched_checkpoint_rejected():
    from paper_1107_4107_b300.api import ArnoldEnsemble, ArnoldError
    X, P = inputs.box(16, seed=26)
    plain = ArnoldEnsemble(16)
    plain.set_state(X, P)
    plain.iterate(20)
    with pytest.raises(ArnoldError):
        plain.indicator("megno")
    with_m = _ens(16)
    with pytest.raises(ArnoldError):
        with_m.restore(plain.checkpoint())
