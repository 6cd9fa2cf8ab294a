"""CUDA adjoint of the N-step map against the oracle's forward-mode gradient and
against central finite differences (the differentiation pattern: gradients of
ensemble observables w.r.t. initial conditions and (h, eps), sqrt(N)
checkpointing with recomputation).

Loss: L = mean_alpha Var_i P_alpha(N) (population variance).  Inputs: the
seeded box X ~ U[0, 2pi)^3, P ~ U([10,11] x [4,5] x [25,26]) (E ~ 390, mostly
regular, so gradients stay finite).  Errors are measured relative to the
largest entry of each gradient.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs

pytestmark = pytest.mark.gpu
H = 0.02 * math.pi


def _ens(n, **kw):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    return ArnoldEnsemble(n, **kw)


def _dl_dp(P):
    n = P.shape[1]
    return (2.0 / 3.0) * (P - P.mean(axis=1, keepdims=True)) / n


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _gpu_grad(X, P, N, C=0, precision="fp64", eps=1.0, h=H):
    ens = _ens(X.shape[1], precision=precision, tangent=False, eps=eps, h=h)
    ens.set_state(X, P)
    ens.forward_ckpt(N, C)
    PN = ens.indicator("P")
    gx, gp, gh, ge = ens.grad(dL_dp=_dl_dp(PN))
    return gx, gp, float(gh), float(ge), PN


@pytest.mark.parametrize("N,n", [(200, 64), (10000, 16)])
def test_fp64_adjoint_matches_oracle_forward_mode(N, n):
    X, P = inputs.box(n, seed=0)
    gx, gp, gh, ge, PN = _gpu_grad(X, P, N)
    ox, op, oh, oe, _, PNo = oracle.gradient(oracle.Params(h=H), X, P, N)
    assert _rel(PN, PNo) < 1e-12
    tol = 1e-9
    assert _rel(gx, ox) < tol and _rel(gp, op) < tol
    assert abs(gh - oh) <= tol * abs(oh) and abs(ge - oe) <= tol * abs(oe)


def test_fp64_adjoint_matches_central_differences():
    """Central differences of L through the CUDA forward map (eta = 1e-6 for the
    initial state, 1e-7 for h and 1e-5 for eps; N = 200), relative error <= 1e-6."""
    n, N = 8, 200
    X, P = inputs.box(n, seed=1)
    gx, gp, gh, ge, _ = _gpu_grad(X, P, N)

    def L(Xi, Pi, eps=1.0, h=H):
        e = _ens(n, tangent=False, eps=eps, h=h)
        e.set_state(Xi, Pi)
        e.iterate(N)
        return float(np.mean(np.var(e.indicator("P"), axis=1)))

    eta = 1e-6
    for a in range(3):
        for i in (0, 5):
            d = np.zeros((3, n)); d[a, i] = eta
            fdx = (L(X + d, P) - L(X - d, P)) / (2 * eta)
            fdp = (L(X, P + d) - L(X, P - d)) / (2 * eta)
            assert abs(fdx - gx[a, i]) <= 1e-6 * np.abs(gx).max()
            assert abs(fdp - gp[a, i]) <= 1e-6 * np.abs(gp).max()
    # parameters: L carries ~1e-14 of FP64 rounding noise, so a 2 * 1e-7 difference
    # resolves dL/deps (~7e-3) only to ~1e-5: eps takes eta = 1e-5.  h moves every
    # angle by ~N |P| eta (5600 eta), so its response is curved on that scale and
    # h takes eta = 1e-7 (noise 5e-8 against dL/dh ~ 6).
    dh, de = 1e-7, 1e-5
    fdh = (L(X, P, h=H + dh) - L(X, P, h=H - dh)) / (2 * dh)
    fde = (L(X, P, eps=1 + de) - L(X, P, eps=1 - de)) / (2 * de)
    assert abs(fdh - gh) <= 1e-6 * abs(gh)
    assert abs(fde - ge) <= 1e-6 * abs(ge)


def test_checkpoint_interval_is_bitwise_invisible():
    X, P = inputs.box(100, seed=2)
    ref = _gpu_grad(X, P, 300, C=1)
    for C in (7, 0, 300):
        got = _gpu_grad(X, P, 300, C=C)
        assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
        assert ref[2] == got[2] and ref[3] == got[3]


def test_fp32c_adjoint_error_vs_fp64_oracle():
    """FP32C recompute + FP32 adjoint: stated bound 1e-4 of the gradient scale at
    N = 200 and 3e-3 at N = 1e4.  The adjoint is a product of 7 N FP32 kick/drift
    Jacobians: a rounding walk of ~6e-8 sqrt(7e4) ~ 1.6e-5, amplified by the
    linear (regular-orbit) growth of the Jacobian over t = 628, gives ~1e-3."""
    for N, n, tol in ((200, 64, 1e-4), (10000, 16, 3e-3)):
        X, P = inputs.box(n, seed=0)
        gx, gp, gh, ge, _ = _gpu_grad(X, P, N, precision="fp32c")
        ox, op, oh, oe, _, _ = oracle.gradient(oracle.Params(h=H), X, P, N)
        errs = (_rel(gx, ox), _rel(gp, op), abs(gh - oh) / abs(oh), abs(ge - oe) / abs(oe))
        print(f"fp32 adjoint N={N}: rel errors x0 {errs[0]:.2e} p0 {errs[1]:.2e} h {errs[2]:.2e} eps {errs[3]:.2e}")
        assert max(errs) < tol, errs


def test_grad_is_repeatable_and_needs_forward():
    from paper_1107_4107_b300._lib import ArnoldError, ESTATE
    X, P = inputs.box(32, seed=3)
    ens = _ens(32, tangent=False)
    ens.set_state(X, P)
    with pytest.raises(ArnoldError) as ex:
        ens.grad(dL_dp=np.ones((3, 32)))
    assert ex.value.status == ESTATE
    ens.forward_ckpt(50)
    a = ens.grad(dL_dp=np.ones((3, 32)))
    b = ens.grad(dL_dp=np.ones((3, 32)))
    assert np.array_equal(a[0], b[0]) and float(a[2]) == float(b[2])
    ens.iterate(1)
    with pytest.raises(ArnoldError):
        ens.grad(dL_dp=np.ones((3, 32)))


def test_autograd_function_variance_loss():
    torch = pytest.importorskip("torch")
    from paper_1107_4107_b300.api import arnold_map
    n, N = 64, 150
    X, P = inputs.box(n, seed=4)
    Xt = torch.tensor(X, device="cuda", requires_grad=True)
    Pt = torch.tensor(P, device="cuda", requires_grad=True)
    h = torch.tensor(H, device="cuda", dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(1.0, device="cuda", dtype=torch.float64, requires_grad=True)
    XN, PN = arnold_map(Xt, Pt, h, eps, N)
    loss = PN.var(dim=1, unbiased=False).mean()
    loss.backward()
    ox, op, oh, oe, _, _ = oracle.gradient(oracle.Params(h=H), X, P, N)
    assert _rel(Xt.grad.cpu().numpy(), ox) < 1e-9
    assert _rel(Pt.grad.cpu().numpy(), op) < 1e-9
    assert abs(h.grad.item() - oh) <= 1e-9 * abs(oh)
    assert abs(eps.grad.item() - oe) <= 1e-9 * abs(oe)


def test_autograd_function_with_float_parameters():
    """h and eps given as plain floats: only X0 and P0 get gradients, and the
    backward pass accepts that (autograd takes no gradient for a non-tensor)."""
    torch = pytest.importorskip("torch")
    from paper_1107_4107_b300.api import arnold_map
    n, N = 64, 150
    X, P = inputs.box(n, seed=4)
    Xt = torch.tensor(X, device="cuda", requires_grad=True)
    Pt = torch.tensor(P, device="cuda", requires_grad=True)
    XN, PN = arnold_map(Xt, Pt, H, 1.0, N)
    loss = PN.var(dim=1, unbiased=False).mean()
    loss.backward()
    ox, op, _, _, _, _ = oracle.gradient(oracle.Params(h=H), X, P, N)
    assert _rel(Xt.grad.cpu().numpy(), ox) < 1e-9
    assert _rel(Pt.grad.cpu().numpy(), op) < 1e-9


def test_sharded_variance_gradient_equals_whole_ensemble():
    """Two shards of one ensemble, each with its own context and CUDA adjoint, run
    the sharded variance-loss gradient (loss partials exchanged before the reverse
    sweep, (h, eps) partials after it) in two host threads with an in-process
    exchange; the result equals the gradient of the whole ensemble."""
    import threading

    from paper_1107_4107_b300 import shard
    from paper_1107_4107_b300.api import ArnoldEnsemble
    n, N, cut = 4096, 200, 1500
    X, P = inputs.box(n, seed=23)
    whole = ArnoldEnsemble(n, tangent=False)
    whole.set_state(X, P)
    whole.forward_ckpt(N)
    PN = whole.indicator("P")
    up = (2.0 / 3.0) * (PN - PN.mean(axis=1, keepdims=True)) / n
    gx, gp, gh, ge = whole.grad(dL_dp=up)

    slots, barrier, results = [None, None], threading.Barrier(2), [None, None]

    def exchange_for(r):
        def ex(obj):
            slots[r] = obj
            barrier.wait()
            out = list(slots)
            barrier.wait()
            return out
        return ex

    def run(r, lo, hi):
        e = ArnoldEnsemble(hi - lo, tangent=False)
        e.set_state(X[:, lo:hi].copy(), P[:, lo:hi].copy())
        e.forward_ckpt(N)
        results[r] = shard.variance_loss_grad(e.indicator("P"), lambda u: e.grad(dL_dp=u), exchange_for(r))
        e.close()

    th = [threading.Thread(target=run, args=(0, 0, cut)), threading.Thread(target=run, args=(1, cut, n))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for r, (lo, hi) in enumerate(((0, cut), (cut, n))):
        L, sgx, sgp, sgh, sge = results[r]
        assert abs(L - float(np.mean(np.var(PN, axis=1)))) <= 1e-13 * L
        np.testing.assert_allclose(sgx, gx[:, lo:hi], rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(sgp, gp[:, lo:hi], rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose([sgh, sge], [float(gh), float(ge)], rtol=1e-12)
