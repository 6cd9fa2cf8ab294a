"""Experiment runners (Fig. 1 sweep, Figs. 2-3 web density, Fig. 4 diffusion) on
small sizes: they run, conserve counts, and a resumed diffusion run equals an
uninterrupted one."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_throughput_sweep_runs():
    from paper_1107_4107_b300.experiments import throughput_vs_n
    rows = throughput_vs_n([1, 148 * 32, 148 * 64 + 1], steps=20)
    assert [r["n"] for r in rows] == [1, 4736, 9473]
    assert all(r["ms"] > 0 for r in rows)


def test_web_density_counts_every_trajectory():
    from paper_1107_4107_b300.experiments import web_density
    r = web_density(20000, 400.0, window_T=2.0, n_cos=32, n_phi=64)
    assert r["counts"].sum() == 20000
    z = web_density(5000, 15.0, window_T=2.0, n_cos=8, n_phi=8, patch=(0.2, 0.45, 0.6, 1.1), track=True)
    assert 0.0 < z["kept_fraction"] <= 1.0
    assert z["counts"].sum() <= 5000


def test_diffusion_resume_equals_uninterrupted(tmp_path):
    from paper_1107_4107_b300.experiments import diffusion_from_w
    kw = dict(n=2000, E=15.0, window_T=1.0, snapshots_T=(2.0, 4.0), n_cos=16, n_phi=16, precision="fp32c")
    full = diffusion_from_w(**kw)
    assert len(full["maps"]) == 2 and all(m["counts"].sum() == 2 * 2000 for m in full["maps"])
    ck = str(tmp_path / "run.ckpt")
    part = diffusion_from_w(**dict(kw, snapshots_T=(2.0,)), ckpt_path=ck)
    rest = diffusion_from_w(**kw, ckpt_path=ck)
    assert np.array_equal(part["maps"][0]["counts"], full["maps"][0]["counts"])
    assert np.array_equal(rest["maps"][0]["counts"], full["maps"][1]["counts"])


def test_scan_agreement_runs_all_modes_from_the_same_ics():
    """The precision-comparison scan: every mode runs from the same grid ICs; the
    FP64 mode is the reference, the others report class agreement and histogram L1
    (short horizon: near-identical classes)."""
    from paper_1107_4107_b300.experiments import scan_agreement
    rows = scan_agreement(E=40.0, steps=300, G=64)
    assert [r["precision"] for r in rows] == ["fp64", "fp32c", "df64", "df64f"]
    for r in rows[1:]:
        assert r["class_agreement"] >= 0.99 and r["hist_l1"] <= 1e-2
    assert all(r["map_steps_per_s"] > 0 for r in rows)
