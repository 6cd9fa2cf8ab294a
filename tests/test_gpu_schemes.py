"""The selectable composition schemes (triple jump, 9 kicks; leapfrog, 1 kick) in
every precision mode and in the adjoint and batched paths, against the oracle
running the same scheme (or, for the batch, bitwise against single ensembles).

Bars: FP64 and the adjoint as for Yoshida-6A (the same arithmetic per kick).
FP32C and DF64 lose accuracy per unit of kick (table sincos and product
roundings), so their 100-step Yoshida bars (3e-7, 3e-11) scale with the total
kick strength sum_k |w_k| of a step relative to Yoshida's 5.71 (triple jump
16.3; leapfrog 1, held at the Yoshida bar), and, as in the full-size test, with
each trajectory's own tangent growth exp(chi t) over the run (first-order error
propagation; these inputs lie near resonances where 100 steps already stretch
errors several-fold)."""
import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs
from parity import oracle_params, rel_err

pytestmark = pytest.mark.gpu

SCHEMES = ["triplejump6", "leapfrog2"]


def _kick_strength(scheme):
    return float(np.sum(np.abs(oracle.scheme_weights(scheme))))


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


@pytest.mark.parametrize("precision,bar", [("fp32c", 3e-7), ("df64", 3e-11), ("df64f", 1e-9)])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_pair_modes_other_schemes_vs_oracle(precision, bar, scheme):
    n, h, R = 333, 0.05, 7
    X, P = inputs.box(n, lo=(-4.0, -4.0, 20.0), hi=(4.0, 4.0, 21.0), seed=51)
    st = oracle.State(X, P, oracle_params(scheme=scheme, h=h, R=R)).advance(100)
    e = _ens(n, precision=precision, scheme=scheme, h=h, renorm_every=R)
    e.set_state(X, P)
    e.iterate(100)
    per_cell = bar * max(1.0, _kick_strength(scheme) / _kick_strength("yoshida6a")) \
        * np.maximum(1.0, np.exp(st.chi() * st.time()))
    for got, ref in ((e.indicator("dX"), st.unwrapped_displacement()), (e.indicator("P"), st.P)):
        err = np.max(np.abs(got - ref) / (1.0 + np.abs(ref)), axis=0)
        assert np.all(err <= per_cell), float(np.max(err / per_cell))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp64_adjoint_other_schemes_vs_oracle(scheme):
    n, N, h = 16, 200, 0.05
    X, P = inputs.box(n, seed=52)
    e = _ens(n, tangent=False, scheme=scheme, h=h)
    e.set_state(X, P)
    e.forward_ckpt(N)
    PN = e.indicator("P")
    up = (2.0 / 3.0) * (PN - PN.mean(axis=1, keepdims=True)) / n
    gx, gp, gh, ge = e.grad(dL_dp=up)
    ox, op, oh, oe, _, PNo = oracle.gradient(oracle.Params(h=h, scheme=scheme), X, P, N)
    assert rel_err(PN, PNo) < 1e-12
    scale = max(np.max(np.abs(ox)), np.max(np.abs(op)))
    assert np.max(np.abs(gx - ox)) <= 1e-9 * scale and np.max(np.abs(gp - op)) <= 1e-9 * scale
    assert abs(float(gh) - oh) <= 1e-9 * abs(oh) and abs(float(ge) - oe) <= 1e-9 * abs(oe)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_batch_other_schemes_bitwise_equal_single(scheme):
    from paper_1107_4107_b300.api import ArnoldBatch
    sets = [{"eps": 1.0, "h": 0.05, "E": 40.0, "G": 24, "n_steps": 300, "seed": 1},
            {"eps": 1.0, "h": 0.0628, "E": 400.0, "G": 13, "n_steps": 77, "seed": 2}]
    b = ArnoldBatch(sets, scheme=scheme)
    R = b.tuning["renorm_every"]
    b.init()
    b.run()
    b.sync()
    for k, q in enumerate(sets):
        e = _ens(q["G"] ** 2, eps=q["eps"], h=q["h"], precision="fp32c", scheme=scheme, renorm_every=R)
        e.init_grid(q["G"], q["E"], seed=q["seed"])
        e.iterate(q["n_steps"])
        for kind in ("X", "P", "tangent", "logsum"):
            assert np.array_equal(b.indicator(k, kind), e.indicator(kind)), (k, kind)
