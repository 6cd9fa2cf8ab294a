"""Compensated-FP32 CUDA path against the FP64 oracle.

FP32C changes the arithmetic (float pairs with TwoSum/TwoProd for angles and
momenta, FP32 forces and tangent), so pointwise agreement is bounded by the
force rounding, not by FP64 rounding: the FP32 table sincos is accurate to
~9e-8 absolute, a kick changes q by at most 2 tau eps ~ 0.17, so each of the
7 kicks of a step adds ~1.5e-8 to the momentum error (abs. ~7e-8 per step
on |P| ~ 28, relative ~2.5e-9 ... 1.2e-8 with the 1 + |P| normalisation of
the smaller components).  Stated bounds on |gpu - oracle| / (1 + |oracle|),
all cells up to 100 steps, and every cell to 1000 times its own tangent growth
G = exp(chi t) from the oracle:
    1 step: 3e-8     100 steps: 3e-7     1000 steps: 3e-6 G
Statistics: the regular/chaotic classes agree on >= 99.5 % of cells and the
histograms of log10 chi differ by <= 1e-2 in L1 (the scan-level tolerances).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_grid_state, oracle_params, rel_err

pytestmark = pytest.mark.gpu

BOUNDS = {1: 3e-8, 100: 3e-7}


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


def test_fp32c_per_step_error_vs_fp64_oracle():
    n = 512
    X, P = inputs.box(n, seed=21)
    st = oracle.State(X, P, oracle_params(R=10))
    ens = _ens(n, precision="fp32c", renorm_every=10)
    ens.set_state(X, P)
    done = 0
    report = {}
    for S in (1, 99, 900):
        ens.iterate(S)
        st.advance(S)
        done += S
        dX = ens.indicator("dX")
        Pg = ens.indicator("P")
        if done in BOUNDS:
            e = max(rel_err(dX, st.unwrapped_displacement()), rel_err(Pg, st.P))
            report[done] = e
            assert e < BOUNDS[done], (done, e)
        else:
            from parity import cell_growth, growth_scaled
            g = cell_growth(st)
            ok1, w1 = growth_scaled(dX, st.unwrapped_displacement(), g, 3e-6)
            ok2, w2 = growth_scaled(Pg, st.P, g, 3e-6)
            report[done] = max(w1, w2)
            assert ok1 and ok2, (done, w1, w2)
    print("fp32c per-step error vs FP64 oracle:", report)


@pytest.mark.parametrize("E", [400.0, 40.0])
def test_fp32c_classification_vs_oracle(E):
    """Config-1 scale horizon (1e4 steps) on a 32 x 32 grid: class agreement with the
    FP64 oracle."""
    G = 32
    ens = _ens(G * G, precision="fp32c")
    ens.init_grid(G, E)
    ens.iterate(10000)
    st = oracle_grid_state(G, E, oracle_params()).advance(10000, threads=8)
    agree = np.mean(ens.indicator("class") == st.classify())
    assert agree >= 0.99, agree


def _l1_hist(a, b):
    ha, _ = np.histogram(np.log10(np.clip(a, 1e-300, None)), bins=200, range=(-8, 1))
    hb, _ = np.histogram(np.log10(np.clip(b, 1e-300, None)), bins=200, range=(-8, 1))
    return float(np.abs(ha / len(a) - hb / len(b)).sum())


@pytest.mark.parametrize("E", [400.0, 40.0])
def test_fp32c_vs_fp64_gpu_scan_agreement(E):
    """128 x 128 grid, 1e4 steps (config 1): FP32C vs FP64 on the GPU, agreement
    >= 99.5 % and histogram L1 <= 1e-2."""
    G = 128
    out = {}
    for prec in ("fp64", "fp32c"):
        ens = _ens(G * G, precision=prec)
        ens.init_grid(G, E)
        ens.iterate(10000)
        out[prec] = (ens.indicator("chi"), ens.indicator("class"))
    agree = np.mean(out["fp64"][1] == out["fp32c"][1])
    l1 = _l1_hist(out["fp64"][0], out["fp32c"][0])
    print(f"E={E}: class agreement {agree:.5f}, hist L1 {l1:.4g}")
    assert agree >= 0.995 and l1 <= 1e-2


def test_fp32c_reduce64_variant_matches(tmp_path):
    """The FP64 mod-2pi reduction variant (ARNOLD_FP32C_REDUCE64=1) agrees with the
    float-pair reduction to FP32C accuracy; run in a child process because the
    switch is read at context creation."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for flag in ("0", "1"):
        path = str(tmp_path / f"r{flag}.npy")
        code = ("import numpy as np; from paper_1107_4107_b300 import inputs; "
                "from paper_1107_4107_b300.api import ArnoldEnsemble as A; X,P=inputs.box(256, seed=3); "
                "e=A(256, precision='fp32c'); e.set_state(X,P); e.iterate(100); "
                f"np.save({path!r}, np.concatenate([e.indicator('dX'), e.indicator('P')]))")
        env = dict(os.environ, ARNOLD_FP32C_REDUCE64=flag, PYTHONPATH=root)
        subprocess.check_call([sys.executable, "-c", code], env=env, cwd=root)
        outs.append(np.load(path))
    assert rel_err(outs[0], outs[1]) < 1e-6


@pytest.mark.parametrize("precision", ["fp32c", "df64", "df64f"])
def test_pair_state_readout_angles_and_energy_error(precision):
    """Pair states hold angles unreduced between exact reductions (FP32C up to 64 rad):
    the read-out must still give X in [0, 2pi) and dE = |H(X, P) - H(X0, P0)| evaluated
    in FP64 from the exported state (identity check of the read-out arithmetic,
    independent of the propagation error)."""
    X0, P0 = inputs.box(300, seed=31)
    ens = _ens(300, precision=precision)
    ens.set_state(X0, P0)
    ens.iterate(150)           # box momenta ~ (10, 4, 25): angles pass 64 rad before the first reduction
    X = ens.indicator("X")
    P = ens.indicator("P")
    assert np.all(X >= 0.0) and np.all(X < 2 * np.pi)
    e0 = oracle.energy(1.0, X0, P0)
    dE_ref = np.abs(oracle.energy(1.0, X, P) - e0)
    assert np.max(np.abs(ens.indicator("dE") - dE_ref)) < 1e-11
    # the unwrapped displacement is unaffected by the read-out reduction
    st = oracle.State(X0, P0, oracle_params()).advance(150)
    assert rel_err(ens.indicator("dX"), st.unwrapped_displacement()) < 3e-6


def test_fp32c_full_size_grid_sampled_cells():
    """The 2048 x 2048 scan in compensated FP32 (default launch configuration):
    256 sampled cells against the FP64 oracle one by one, 100 steps.  The grid holds
    cells near resonances where the flow already stretches errors within 100 steps, so
    each cell's bar is the 100-step bound times its own tangent growth
    |w(t)| / |w(0)| = exp(chi t) from the oracle (first-order error propagation)."""
    G, E = 2048, 400.0
    ens = _ens(G * G, precision="fp32c")
    ens.init_grid(G, E)
    ens.iterate(100)
    cells = inputs.sample_cells(G * G, 256, seed=4)
    st = oracle_grid_state(G, E, oracle_params(), cells=cells).advance(100, threads=4)
    growth = np.exp(st.chi() * st.time())
    bar = BOUNDS[100] * np.maximum(1.0, growth)
    for got, ref in ((ens.indicator("dX")[:, cells], st.unwrapped_displacement()),
                     (ens.indicator("P")[:, cells], st.P)):
        err = np.max(np.abs(got - ref) / (1.0 + np.abs(ref)), axis=0)
        k = int(np.argmax(err / bar))
        print(f"worst cell: err {err[k]:.2e}, growth {growth[k]:.2f}, bar {bar[k]:.2e}")
        assert np.all(err <= bar)


def test_fp32c_range_is_reported():
    """FP32C holds angles in a [1024, 2048) rad window, valid while an angle moves
    at most 400 rad per step (h |q| <= 400): beyond that the run reports ERANGE at
    the next renormalisation (the table index stays masked, so nothing is read out
    of bounds meanwhile)."""
    from paper_1107_4107_b300._lib import ERANGE
    from paper_1107_4107_b300.api import ArnoldError
    X, P = inputs.box(64, seed=61)
    P[0] *= 50.0                          # |q| ~ 500 at h = 1: 500 rad per step
    e = _ens(64, precision="fp32c", h=1.0, renorm_every=5)
    e.set_state(X, P)
    e.iterate(10)
    with pytest.raises(ArnoldError) as ex:
        e.sync()
    assert ex.value.status == ERANGE
    ok = _ens(64, precision="fp32c", h=0.05, renorm_every=5)
    ok.set_state(*inputs.box(64, seed=61))
    ok.iterate(10)
    ok.sync()
