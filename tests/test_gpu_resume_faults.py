"""Checkpoint/resume (bitwise continuation) and failure handling without any
GPU fault: host-injected errors (ARNOLD_FAULT) and a non-finite state detected
by the kernels' own checks, after which the context stays usable."""
import os

import numpy as np
import pytest

from paper_1107_4107_b300 import inputs
from paper_1107_4107_b300._lib import ArnoldError, ECUDA, EINVAL, ENONFINITE, ETIMEOUT

pytestmark = pytest.mark.gpu
KINDS = ("X", "P", "dX", "tangent", "chi", "V", "dE_max", "logsum")


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_resume_is_bitwise(precision, tmp_path):
    n = 3000
    X, P = inputs.box(n, seed=31)
    kw = dict(precision=precision, renorm_every=7, window=40)
    ref = _ens(n, **kw)
    ref.set_state(X, P)
    ref.iterate(333)
    a = _ens(n, **kw)
    a.set_state(X, P)
    a.iterate(150)
    path = str(tmp_path / "state.ckpt")
    a.save(path)
    a.close()
    b = _ens(n, **kw)
    b.load(path)
    assert b.steps == 150
    b.iterate(183)
    for k in KINDS:
        assert np.array_equal(ref.indicator(k), b.indicator(k)), k


def test_checkpoint_rejects_mismatched_context():
    a = _ens(100)
    a.set_state(*inputs.box(100, seed=1))
    blob = a.checkpoint()
    for kw in ({"precision": "fp32c"}, {"h": 0.05}, {"tangent": False}):
        with pytest.raises(ArnoldError) as e:
            _ens(100, **kw).restore(blob)
        assert e.value.status == EINVAL
    with pytest.raises(ArnoldError):
        _ens(101).restore(blob + b"\0")
    bad = bytearray(blob)
    bad[0:8] = b"XXXXXXXX"
    with pytest.raises(ArnoldError):
        _ens(100).restore(bytes(bad))


def test_injected_faults_propagate_and_context_survives(monkeypatch):
    e = _ens(64)
    e.set_state(*inputs.box(64, seed=2))
    for fault, call, status in (("launch", lambda: e.iterate(5), ECUDA), ("timeout", e.sync, ETIMEOUT),
                                ("nan", lambda: e.indicator("P"), ENONFINITE)):
        monkeypatch.setenv("ARNOLD_FAULT", fault)
        with pytest.raises(ArnoldError) as ex:
            call()
        assert ex.value.status == status
        monkeypatch.delenv("ARNOLD_FAULT")
        e.iterate(3)
        e.sync()
    assert np.all(np.isfinite(e.indicator("P")))
    e.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_nonfinite_state_is_reported_not_trapped(precision):
    """A NaN momentum is carried, found at the next renormalisation, and reported
    as ENONFINITE by sync; a fresh state then runs normally on the same context."""
    n = 128
    X, P = inputs.box(n, seed=3)
    P[0, 5] = np.nan
    e = _ens(n, precision=precision, renorm_every=5)
    e.set_state(X, P)
    e.iterate(10)
    with pytest.raises(ArnoldError) as ex:
        e.sync()
    assert ex.value.status == ENONFINITE
    X, P = inputs.box(n, seed=4)
    e.set_state(X, P)
    e.iterate(10)
    e.sync()
    assert np.all(np.isfinite(e.indicator("chi")))
