"""Batched persistent launch (many (K, eps) sets of uneven sizes and step counts,
one CUDA-graph launch, FP32C or double-float): every set must be bit-identical
to a single ensemble of the same precision with the same parameters, for any
tuning, across repeated runs.  The single ensembles are themselves held to the
oracle by the per-precision parity tests."""
import numpy as np
import pytest

from paper_1107_4107_b300 import params

pytestmark = pytest.mark.gpu

SETS = [
    {"eps": 1.0, "h": 0.0628, "E": 400.0, "G": 17, "n_steps": 150, "seed": 1},
    {"eps": 1.0, "h": 0.05, "E": 40.0, "G": 32, "n_steps": 1000, "seed": 2},
    {"eps": 0.5, "h": 0.1, "E": 2000.0, "G": 45, "n_steps": 37, "seed": 3},
    {"eps": 1.0, "h": 0.0314, "E": 20.0, "G": 64, "n_steps": 500, "seed": 4},
    {"eps": 1.0, "h": 0.1257, "E": 200000.0, "G": 8, "n_steps": 2000, "seed": 5},
    {"eps": 2.0, "h": 0.07, "E": 15.0, "G": 100, "n_steps": 300, "seed": 6},
]
KINDS = ("X", "P", "dX", "tangent", "chi", "dE_max", "logsum")


def _single(q, steps_list, R, precision):
    from paper_1107_4107_b300.api import ArnoldEnsemble
    e = ArnoldEnsemble(q["G"] ** 2, eps=q["eps"], h=q["h"], precision=precision, renorm_every=R)
    e.init_grid(q["G"], q["E"], seed=q["seed"])
    for s in steps_list:
        e.iterate(s)
    out = {k: e.indicator(k) for k in KINDS}
    e.sync()
    return out


@pytest.mark.parametrize("precision,tuning", [
    ("fp32c", None),
    ("fp32c", {"block_size": 128, "traj_per_thread": 2, "renorm_every": 50, "epoch_ms": 5}),
    ("df64f", None),
    ("df64f", {"block_size": 128, "traj_per_thread": 1, "renorm_every": 50, "epoch_ms": 5}),
    ("df64", {"block_size": 64, "traj_per_thread": 1, "renorm_every": 100, "epoch_ms": 5}),
])
def test_batch_bitwise_equals_single_ensembles(precision, tuning):
    from paper_1107_4107_b300.api import ArnoldBatch
    b = ArnoldBatch(SETS, tuning=tuning, precision=precision)
    R = b.tuning["renorm_every"]
    b.init()
    b.run()
    b.run()       # a replay continues every set
    b.sync()
    info = b.info()
    assert info["map_steps_per_run"] == sum(q["G"] ** 2 * q["n_steps"] for q in SETS)
    assert info["epochs"] >= 1
    for k, q in enumerate(SETS):
        ref = _single(q, [q["n_steps"], q["n_steps"]], R, precision)
        for kind in KINDS:
            assert np.array_equal(b.indicator(k, kind), ref[kind]), (k, kind)


def test_batch_double_float_rejects_two_per_thread():
    from paper_1107_4107_b300._lib import ArnoldError, EINVAL
    from paper_1107_4107_b300.api import ArnoldBatch
    with pytest.raises(ArnoldError) as ex:
        ArnoldBatch(SETS[:2], precision="df64f", tuning={"block_size": 128, "traj_per_thread": 2,
                                                         "renorm_every": 100, "epoch_ms": 5})
    assert ex.value.status == EINVAL
    with pytest.raises(ArnoldError) as ex:
        ArnoldBatch(SETS[:2], precision="fp64")
    assert ex.value.status == EINVAL


def test_batch_plan_for_the_batched_scan_config():
    """The 64-set (K, eps_eff) grid: plan sizes and one short run (steps / 1000)."""
    from paper_1107_4107_b300.api import ArnoldBatch
    sets = params.batch_sets(step_scale=1e-3)
    b = ArnoldBatch(sets)
    b.init()
    b.run()
    b.sync()
    info = b.info()
    assert info["map_steps_per_run"] == sum(q["G"] ** 2 * q["n_steps"] for q in sets)
    for k in (0, 31, 63):
        s = b.stats(k)
        assert s["n"] == sets[k]["G"] ** 2


@pytest.mark.parametrize("precision", ["fp32c", "df64f"])
def test_autotuner_picks_and_caches(tmp_path, monkeypatch, precision):
    from paper_1107_4107_b300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    cands = [{"block_size": 128, "traj_per_thread": 1, "renorm_every": 100, "epoch_ms": 50},
             {"block_size": 256, "traj_per_thread": 1, "renorm_every": 100, "epoch_ms": 50}]
    best = tune.tune_batch(SETS, candidates=cands, precision=precision)
    assert best in cands
    assert tune.tune_batch(SETS, candidates=cands, precision=precision) == best      # from the cache
    assert (tmp_path / "cache.json").exists()


@pytest.mark.parametrize("precision", ["df64f", "fp32c"])
def test_batch_degenerate_sets_and_no_tangent(precision):
    """Degenerate sets in one batch: a 1 x 1 grid, a set with zero steps (left
    untouched), a ragged 3 x 3 grid, with the tangent off; each still equals its
    single ensemble bit for bit, and the zero-step set keeps its initial state."""
    from paper_1107_4107_b300.api import ArnoldBatch, ArnoldEnsemble
    sets = [{"eps": 1.0, "h": 0.0628, "E": 400.0, "G": 1, "n_steps": 77, "seed": 11},
            {"eps": 1.0, "h": 0.05, "E": 40.0, "G": 16, "n_steps": 0, "seed": 12},
            {"eps": 1.0, "h": 0.1257, "E": 200000.0, "G": 3, "n_steps": 513, "seed": 13}]
    b = ArnoldBatch(sets, tangent=False, precision=precision,
                    tuning={"block_size": 64, "traj_per_thread": 1, "renorm_every": 50, "epoch_ms": 5})
    b.init()
    b.run()
    b.sync()
    assert b.info()["map_steps_per_run"] == 77 + 0 + 9 * 513
    for k, q in enumerate(sets):
        e = ArnoldEnsemble(q["G"] ** 2, eps=q["eps"], h=q["h"], precision=precision, tangent=False,
                           renorm_every=50)
        e.init_grid(q["G"], q["E"], seed=q["seed"])
        if q["n_steps"]:
            e.iterate(q["n_steps"])
        for kind in ("X", "P", "dE_max"):
            assert np.array_equal(b.indicator(k, kind), e.indicator(kind)), (k, kind)
    assert np.array_equal(b.indicator(1, "dE_max"), np.zeros(256))
