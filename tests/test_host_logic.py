"""Host-side logic on CPU: parameter plumbing, batched-scan set generator, shard
layout, statistics merging, and the two-rank merge over torch.distributed (gloo)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1107_4107_b300 import inputs, params, shard


def test_parameter_conversions():
    assert params.eps_eff(400.0) == 0.005
    assert abs(params.energy_for(params.eps_eff(15.0)) - 15.0) < 1e-12
    h = params.paper_h()
    K = params.kick_strength(1.0, h)
    assert abs(params.h_for(K) - h) < 1e-15
    # chain rule h = sqrt(K / eps): compare with finite differences of a smooth f(h, eps)
    f = lambda hh, ee: math.sin(hh * 3.0) + ee ** 2 * hh          # noqa: E731
    g_h = 3.0 * math.cos(h * 3.0) + 1.0 ** 2
    g_e = 2.0 * 1.0 * h
    dK, de = params.grads_K_eps(g_h, g_e, h, 1.0)
    d = 1e-7
    fK = lambda KK, ee: f(math.sqrt(KK / ee), ee)                   # noqa: E731
    assert abs((fK(K + d, 1.0) - fK(K - d, 1.0)) / (2 * d) - dK) < 1e-6 * abs(dK)
    assert abs((fK(K, 1.0 + d) - fK(K, 1.0 - d)) / (2 * d) - de) < 1e-6 * max(1, abs(de))


def test_batch_sets_generator():
    s = params.batch_sets()
    assert len(s) == 64
    ee = sorted({q["eps_eff"] for q in s})
    KK = sorted({q["K"] for q in s})
    assert len(ee) == 8 and len(KK) == 8
    assert abs(ee[0] - 1e-5) < 1e-18 and abs(ee[-1] - 0.1) < 1e-15
    assert abs(KK[0] - (0.005 * 2 * math.pi) ** 2) < 1e-15 and abs(KK[-1] - (0.02 * 2 * math.pi) ** 2) < 1e-15
    for q in s:
        assert 1e3 * 0.8 <= q["G"] ** 2 <= 1e6 * 1.01 and 1e4 <= q["n_steps"] <= 1e6
        assert abs(q["E"] - 2.0 / q["eps_eff"]) < 1e-9 * q["E"]
        assert abs(q["h"] ** 2 - q["K"]) < 1e-15
    assert s == params.batch_sets()             # seeded, reproducible


@pytest.mark.parametrize("G,world", [(2048, 1), (2048, 3), (17, 4), (5, 5)])
def test_row_bands_partition_the_grid(G, world):
    bands = [shard.row_band(G, r, world) for r in range(world)]
    assert bands[0][0] == 0
    for (r0, n0), (r1, _) in zip(bands, bands[1:]):
        assert r0 + n0 == r1
    assert sum(n for _, n in bands) == G
    assert max(n for _, n in bands) - min(n for _, n in bands) <= 1


def _synthetic(n, seed):
    rng = np.random.default_rng(seed)
    chi = 10.0 ** rng.uniform(-9, 2, n)
    dE = rng.uniform(0, 1e-3, n)
    P = rng.normal(size=(3, n)) * [[1.0], [2.0], [3.0]] + [[5.0], [0.0], [-2.0]]
    return chi, dE, P


def test_merge_stats_equals_unsharded():
    chi, dE, P = _synthetic(10001, 1)
    t = 628.3
    whole = oracle.stats(chi, dE, P, t)
    cuts = [0, 17, 5000, 5001, 10001]
    parts = []
    for a, b in zip(cuts, cuts[1:]):
        p = oracle.stats(chi[a:b], dE[a:b], P[:, a:b], t)
        p["n"] = b - a
        parts.append(p)
    m = shard.merge_stats(parts)
    assert np.array_equal(m["hist"], whole["hist"])
    for k in ("under", "over", "chaotic"):
        assert m[k] == whole[k]
    assert m["dE_max"] == whole["dE_max"]
    np.testing.assert_allclose(m["p_mean"], whole["p_mean"], rtol=1e-12)
    np.testing.assert_allclose(m["p_var"], whole["p_var"], rtol=1e-12)


def _rank_main(rank, world, port, n, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    chi, dE, P = _synthetic(n, 7)
    r0, rows = shard.row_band(n, rank, world)
    part = oracle.stats(chi[r0:r0 + rows], dE[r0:r0 + rows], P[:, r0:r0 + rows], 100.0)
    part["n"] = rows
    merged = shard.gather_stats(part)
    if rank == 0:
        np.save(out_path, np.concatenate([merged["hist"], [merged["under"], merged["over"], merged["chaotic"],
                                                            merged["n"]], merged["p_mean"], merged["p_var"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge(tmp_path):
    """World size 2 over gloo on CPU: each rank reduces its band, the merged
    statistics equal those of the whole ensemble."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    n = 4001
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, port, n, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    chi, dE, P = _synthetic(n, 7)
    whole = oracle.stats(chi, dE, P, 100.0)
    nb = len(whole["hist"])
    assert np.array_equal(got[:nb], whole["hist"])
    assert list(got[nb:nb + 4]) == [whole["under"], whole["over"], whole["chaotic"], n]
    np.testing.assert_allclose(got[nb + 4:nb + 7], whole["p_mean"], rtol=1e-12)
    np.testing.assert_allclose(got[nb + 7:nb + 10], whole["p_var"], rtol=1e-12)


def _adjoint_case():
    X, P = inputs.box(24, seed=17)
    prm = oracle.Params(renorm_every=100)
    return prm, X, P, 40


def _adjoint_rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prm, X, P, N = _adjoint_case()
    r0, cnt = shard.row_band(X.shape[1], rank, world)
    Xl, Pl = X[:, r0:r0 + cnt], P[:, r0:r0 + cnt]
    PN = oracle.State(Xl, Pl, prm, tangent=False).advance(N).P

    def local_backward(up):
        gx, gp, gh, ge, _, _ = oracle.gradient(prm, Xl, Pl, N, dL_dpN=up)
        return gx, gp, gh, ge

    L, gx, gp, gh, ge = shard.variance_loss_grad(PN, local_backward, shard.dist_exchange())
    np.save(out_path + f".{rank}.npy", np.concatenate([[L, gh, ge], gx.ravel(), gp.ravel()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharded_adjoint(tmp_path):
    """World size 2 over gloo on CPU: the sharded variance-loss gradient (loss
    partials exchanged before the reverse sweep, (h, eps) partials after it), with
    the oracle's forward-mode gradient as each rank's local backward, equals the
    oracle gradient of the whole ensemble."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "adj")
    mp.start_processes(_adjoint_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    prm, X, P, N = _adjoint_case()
    gx, gp, gh, ge, _, PN = oracle.gradient(prm, X, P, N)
    L = oracle.loss_variance(PN)
    for rank in range(2):
        r0, cnt = shard.row_band(X.shape[1], rank, 2)
        got = np.load(out + f".{rank}.npy")
        np.testing.assert_allclose(got[:3], [L, gh, ge], rtol=1e-12)
        np.testing.assert_allclose(got[3:3 + 3 * cnt].reshape(3, cnt), gx[:, r0:r0 + cnt], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(got[3 + 3 * cnt:].reshape(3, cnt), gp[:, r0:r0 + cnt], rtol=1e-12, atol=1e-15)


def test_sharded_loss_merge_any_split():
    """Loss partials merged in rank order give the whole ensemble's mean, variance
    and loss for uneven splits, including an empty shard."""
    rng = np.random.default_rng(5)
    P = rng.normal(10.0, 3.0, (3, 1001))
    whole = shard.combine_loss([shard.loss_partials(P)])
    for cuts in ([0, 1, 500, 1001], [0, 0, 1001], [0, 333, 334, 1001]):
        parts = [shard.loss_partials(P[:, a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
        c = shard.combine_loss(parts)
        assert c["n"] == 1001
        np.testing.assert_allclose(c["mean"], whole["mean"], rtol=1e-14)
        np.testing.assert_allclose(c["var"], whole["var"], rtol=1e-12)
        assert abs(c["loss"] - oracle.loss_variance(P)) <= 1e-12 * abs(c["loss"])


def test_arnold_map_is_one_autograd_function():
    """ArnoldMap is a single module-level torch.autograd.Function (built once, on
    first use) and arnold_map applies it."""
    torch = pytest.importorskip("torch")
    from paper_1107_4107_b300 import api
    F = api.ArnoldMap
    assert issubclass(F, torch.autograd.Function)
    assert api.ArnoldMap is F
    with pytest.raises(AttributeError):
        api.NoSuchName  # noqa: B018


class _OracleBand:
    """Stand-in for ArnoldEnsemble on the CPU (the oracle), holding one band of
    rows of a grid scan, with the calls bench.bench_step makes."""

    def __init__(self, G, E, row0, rows, seed):
        X, Pxy = inputs.grid_slice(G, E, 1.0, seed=seed, rows=(row0, row0 + rows))
        P = np.zeros((3, X.shape[1]))
        P[:2] = Pxy
        self.st = oracle.State(X, oracle.pz_from_energy(E, 1.0, X, P), oracle.Params())

    def iterate(self, k):
        self.st.advance(k)

    def indicator(self, kind, out):
        val = {"chi": self.st.chi, "class": self.st.classify, "V": self.st.velocity,
               "dE_max": lambda: self.st.dE_max}[kind]()
        out[...] = val

    def stats(self):
        s = oracle.stats(self.st.chi(), self.st.dE_max, self.st.P, self.st.time())
        s["n"] = self.st.n
        return s


def _bench_band_rank(rank, world, port, out_path, G, E, chunk):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    row0, rows, seed = bench.rank_workload(world, rank, "band", grid=G)
    ens = _OracleBand(G, E, row0, rows, seed)
    n = rows * G
    outs = {"chi": np.empty(n), "class": np.empty(n, dtype=np.uint8), "V": np.empty((3, n)), "dE_max": np.empty(n)}
    bench.bench_step(ens, chunk, outs, gather=None)          # a first chunk without exchange
    merged = bench.bench_step(ens, chunk, outs, gather=shard.gather_stats)
    if rank == 0:
        np.save(out_path, np.concatenate([merged["hist"], [merged["under"], merged["over"], merged["chaotic"],
                                                            merged["n"], merged["dE_max"]],
                                          merged["p_mean"], merged["p_var"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_banded_scan_on_two_gloo_ranks(tmp_path):
    """The bench's N > 1 path (rank_workload's row bands, bench_step's statistics
    merge over the process group) on two CPU ranks with the oracle in place of the
    GPU ensemble: the merged statistics of the banded scan equal those of the
    whole scan run in one piece."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    G, E, chunk = 15, 40.0, 60
    out = str(tmp_path / "band.npy")
    mp.start_processes(_bench_band_rank, args=(2, port, out, G, E, chunk), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    whole = _OracleBand(G, E, 0, G, 0)
    whole.iterate(2 * chunk)
    ref = whole.stats()
    nb = len(ref["hist"])
    assert np.array_equal(got[:nb], ref["hist"])
    assert list(got[nb:nb + 4]) == [ref["under"], ref["over"], ref["chaotic"], G * G]
    assert got[nb + 4] == ref["dE_max"]
    np.testing.assert_allclose(got[nb + 5:nb + 8], ref["p_mean"], rtol=1e-12)
    np.testing.assert_allclose(got[nb + 8:nb + 11], ref["p_var"], rtol=1e-12)


class _BlobEnsemble:
    """Stand-in with the checkpoint calls of ArnoldEnsemble (host logic only)."""

    def __init__(self, blob=b""):
        self.blob = blob

    def checkpoint(self):
        return self.blob

    def restore(self, blob):
        self.blob = blob


def test_fig4_checkpoint_is_one_atomic_file_checked_on_resume(tmp_path):
    """The Fig. 4 runner's checkpoint holds state, window count and accumulated F
    in one file written by rename; resuming checks F against the windows done
    since the last snapshot boundary and refuses anything else."""
    from paper_1107_4107_b300.experiments import _load_fig4_ckpt, _save_fig4_ckpt
    path = str(tmp_path / "fig4.ckpt")
    bounds, shape = [2, 10], (4, 8)
    acc = np.zeros(shape, dtype=np.int64)
    acc[1, 2] = 7
    _save_fig4_ckpt(path, _BlobEnsemble(b"state-after-5-windows"), 5, acc)
    assert sorted(os.listdir(tmp_path)) == ["fig4.ckpt"]          # no temporary left behind
    e = _BlobEnsemble()
    done, got = _load_fig4_ckpt(path, e, bounds, shape)
    assert done == 5 and np.array_equal(got, acc) and e.blob == b"state-after-5-windows"
    for bad_done, bad_acc, bad_shape in ((5, np.zeros(shape), shape),       # windows 3-5 missing from F
                                         (2, acc, shape),                   # F not empty at a boundary
                                         (5, acc, (8, 4))):                 # another F grid
        _save_fig4_ckpt(path, _BlobEnsemble(b"x"), bad_done, np.asarray(bad_acc))
        with pytest.raises(ValueError):
            _load_fig4_ckpt(path, _BlobEnsemble(), bounds, bad_shape)
    np.savez(path + ".npz", state=np.zeros(3, np.uint8))           # not a Fig. 4 checkpoint
    with pytest.raises(ValueError):
        _load_fig4_ckpt(path + ".npz", _BlobEnsemble(), bounds, shape)


def test_tuner_candidates_per_precision():
    from paper_1107_4107_b300 import tune
    assert any(c["traj_per_thread"] == 2 for c in tune.candidates_for("fp32c"))
    for prec in ("df64f", "df64"):
        c = tune.candidates_for(prec)
        assert c and all(x["traj_per_thread"] == 1 for x in c)


def test_bench_workload_per_rank():
    """Bands cover the scan's rows once (strong scaling); independent mode gives
    every rank the whole grid with its own seed (weak scaling)."""
    import bench
    rows = [bench.rank_workload(4, r, "band", grid=2048) for r in range(4)]
    assert [r0 for r0, _, _ in rows] == [0, 512, 1024, 1536] and {s for _, _, s in rows} == {0}
    assert sum(n for _, n, _ in rows) == 2048
    assert [bench.rank_workload(3, r, "independent", grid=2048) for r in range(3)] == [(0, 2048, r) for r in range(3)]


def test_long_horizon_oracle_records_describe_the_sampled_cells():
    """The oracle's 1e6-step records (tests/golden/oracle_scan_2048_1e6*.json)
    hold, for every energy the GPU test compares, chi at every mark on exactly
    the cells the seeded sampler draws; the one-ulp record has the same cells."""
    import hashlib
    import json
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(here, "oracle_scan_2048_1e6.json")) as f:
        g = json.load(f)
    with open(os.path.join(here, "oracle_scan_2048_1e6_ulp.json")) as f:
        u = json.load(f)
    idx = inputs.sample_cells(g["grid"] ** 2, g["cells"], seed=g["sample_seed"])
    assert hashlib.sha256(idx.astype("<i8").tobytes()).hexdigest() == g["cells_sha256"]
    for key in ("grid", "eps", "h", "renorm_every", "seed", "sample_seed", "cells", "cells_sha256", "marks"):
        assert u[key] == g[key], key
    assert set(g["energies"]) == {"400", "40", "15"}
    assert set(u["energies"]) == {"40", "15"}
    for rec in (g, u):
        for row in rec["energies"].values():
            assert set(row["chi"]) == {str(m) for m in g["marks"]}
            for chi in row["chi"].values():
                chi = np.asarray(chi)
                assert chi.shape == (g["cells"],) and np.all(np.isfinite(chi)) and np.all(chi > 0)


def test_long_horizon_record_merge_refuses_other_cells(tmp_path):
    """make_oracle_scan_1e6.py --energy adds an energy to an existing record
    only if that record describes the same grid, cells and marks."""
    import importlib.util
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_oracle_scan_1e6.py")
    spec = importlib.util.spec_from_file_location("make_oracle_scan_1e6", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    base = {"grid": 2048, "eps": 1.0, "h": 0.1, "renorm_every": 100, "scheme": "yoshida6a", "seed": 0,
            "sample_seed": 2048, "cells": 4, "cells_sha256": "abc", "marks": [10, 100], "energies": {}}
    out = str(tmp_path / "rec.json")
    assert mod._merge_base(dict(base), out) == base            # nothing stored yet: the new record
    stored = dict(base, energies={"400": {"chi": {}}})
    with open(out, "w") as f:
        json.dump(stored, f)
    assert mod._merge_base(dict(base), out)["energies"] == {"400": {"chi": {}}}
    with pytest.raises(SystemExit):
        mod._merge_base(dict(base, cells_sha256="def"), out)
    with pytest.raises(SystemExit):
        mod._merge_base(dict(base, marks=[10, 1000]), out)


def test_binding_checks_caller_buffers_before_the_library_sees_them():
    """The C ABI takes bare pointers, so the binding checks every caller buffer's
    element count, dtype, host/device kind and device first: a bad one raises
    ValueError and never reaches the library; a good one does (here the library
    then refuses the NULL context with EINVAL, as no GPU is needed for that)."""
    torch = pytest.importorskip("torch")
    from paper_1107_4107_b300 import _lib
    from paper_1107_4107_b300.api import ArnoldBatch, ArnoldEnsemble, _buf
    n = 16
    e = object.__new__(ArnoldEnsemble)
    e.n, e.device, e._h = n, 0, None
    bad = [lambda: e.indicator("chi", out=np.empty(n - 1)),                       # short
           lambda: e.indicator("chi", out=np.empty(n, dtype=np.float32)),         # mistyped
           lambda: e.indicator("class", out=np.empty(n)),                         # u8 kind into f64
           lambda: e.indicator("V", out=np.empty(n)),                             # [3][n] kind
           lambda: e.init_grid(4, 400.0, raw_out=np.empty((6, n))),               # host memory for a device write
           lambda: e.init_grid(4, 400.0, raw_out=torch.empty((6, n), dtype=torch.float64)),
           lambda: e.set_state_shell(np.zeros((3, n)), np.zeros((2, n)), 2, 400.0),
           lambda: e.velocity_histogram(4, 8, out=np.zeros((4, 7), dtype=np.uint64)),
           lambda: e.velocity_histogram(4, 8, out=np.zeros((4, 8))),
           lambda: e.stats_arrays(np.zeros(n), np.zeros(n), np.zeros((3, n)), 1.0),   # device arrays only
           lambda: e.grad(dL_dp=np.ones((3, n - 1))),
           lambda: e.grad(dL_dp=np.ones((3, n)), out_x=np.empty((3, n)), out_p=np.empty((2, n))),
           lambda: e.grad(dL_dp=np.ones((3, 2 * n))[:, ::2])]                         # not contiguous
    for call in bad:
        with pytest.raises(ValueError):
            call()
    good = [lambda: e.indicator("chi", out=np.empty(n)),
            lambda: e.indicator("class", out=torch.empty(n, dtype=torch.uint8)),
            lambda: e.indicator("V", out=np.empty((3, n))),
            lambda: e.set_state_shell(np.zeros((3, n)), np.zeros((3, n)), 2, 400.0),
            lambda: e.velocity_histogram(4, 8, out=np.zeros((4, 8), dtype=np.uint64)),
            lambda: e.velocity_histogram(4, 8, out=torch.zeros((4, 8), dtype=torch.int64)),
            lambda: e.grad(dL_dp=np.ones((3, n)))]
    for call in good:
        with pytest.raises(_lib.ArnoldError) as ex:
            call()
        assert ex.value.status == _lib.EINVAL
    b = object.__new__(ArnoldBatch)
    b.sets, b.device, b._h = [{"G": 4}], 0, None
    with pytest.raises(ValueError):
        b.indicator(0, "chi", out=np.empty(15))
    with pytest.raises(_lib.ArnoldError):
        b.indicator(0, "chi", out=np.empty(16))
    assert _buf(np.empty((2, 3)), 6, ("float64",), "a", 0)[1] == _lib.HOST
