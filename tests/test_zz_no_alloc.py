"""The allocation-free statistics entry point against the regular one.

arnold_stats_arrays_noalloc serves callers that cannot call cudaMalloc (a
framework's caching allocator holds the memory, device-wide synchronisation is
not allowed, or the memory budget is fixed): its reduction scratch is a fixed
array inside the library.  This test calls it through the C ABI twice in a row
on different inputs and checks each result against arnold_stats_arrays on the
same inputs: counts and the maximum exactly, moments to 1e-12 (the partials
are merged in a different grouping, so only rounding may differ).  It lives in
a file collected last so that a stop-at-first-failure run has already run the
rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_1107_4107_b300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _arrays(torch, n, seed):
    r = inputs.uniform01(inputs.splitmix64(seed, np.arange(5 * n, dtype=np.uint64))).reshape(5, n)
    chi = 10.0 ** (-9.0 + 11.0 * r[0])
    chi[:3] = [0.0, -2.0, 1e-3]
    dE = 1e-4 * r[1]
    P = np.stack([20 * r[2] - 10, 5 * r[3] + 2, r[4] - 0.5])
    dev = lambda a: torch.tensor(a, device="cuda", dtype=torch.float64)  # noqa: E731
    return dev(chi), dev(dE), dev(np.ascontiguousarray(P))


def _noalloc(torch, chi, dE, P, t):
    s = _lib.Stats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().arnold_stats_arrays_noalloc(0, stream, int(chi.shape[0]), ctypes.c_void_p(chi.data_ptr()),
                                                ctypes.c_void_p(dE.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                                t, 10.0, ctypes.byref(s))
    _lib.check(rc, "arnold_stats_arrays_noalloc")
    from paper_1107_4107_b300.api import stats_dict
    return stats_dict(s)


def test_noalloc_stats_match_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_1107_4107_b300.api import ArnoldEnsemble
    ens = ArnoldEnsemble(8)
    for n, seed, t in ((1_000_003, 41, 628.3185307179587), (70_001, 42, 6283.185307179586)):
        chi, dE, P = _arrays(torch, n, seed)
        before = torch.cuda.current_device()
        got = _noalloc(torch, chi, dE, P, t)
        assert torch.cuda.current_device() == before     # the caller's device is left as it was
        ref = ens.stats_arrays(chi, dE, P, t)
        assert got["n"] == ref["n"] == n
        assert np.array_equal(got["hist"], ref["hist"])
        for k in ("under", "over", "chaotic"):
            assert got[k] == ref[k], k
        assert got["dE_max"] == ref["dE_max"]
        np.testing.assert_allclose(got["p_mean"], ref["p_mean"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got["p_var"], ref["p_var"], rtol=1e-12)


def test_noalloc_rejects_sizes_beyond_the_limit():
    s = _lib.Stats()
    one = ctypes.c_void_p(1)
    rc = _lib.lib().arnold_stats_arrays_noalloc(0, None, _lib.NOALLOC_MAX_N + 1, one, one, one, 1.0, 10.0,
                                                ctypes.byref(s))
    assert rc == _lib.EINVAL
