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


def test_scan_one_ulp_fp64_arm():
    """The "fp64ulp" arm of the scan: FP64 from the grid's angles moved up by one
    ulp, p_z again from the energy (the same perturbation as the oracle's one-ulp
    record).  Over a short horizon its classes agree with FP64's, and it starts
    from a moved state on the energy shell."""
    import torch

    import oracle
    from paper_1107_4107_b300.api import ArnoldEnsemble
    from paper_1107_4107_b300.experiments import scan_agreement
    rows = scan_agreement(E=15.0, steps=300, G=64, precisions=("fp64", "fp64ulp"))
    assert [r["precision"] for r in rows] == ["fp64", "fp64ulp"]
    assert rows[1]["class_agreement"] >= 0.99 and rows[1]["hist_l1"] <= 1e-2
    G, E = 64, 15.0
    raw = torch.empty((6, G * G), dtype=torch.float64, device="cuda:0")
    a = ArnoldEnsemble(G * G, precision="fp64")
    a.init_grid(G, E, raw_out=raw)
    a.sync()
    X = torch.nextafter(raw[:3], torch.full_like(raw[:3], math.inf)).contiguous()
    b = ArnoldEnsemble(G * G, precision="fp64")
    b.set_state_shell(X, raw[3:].contiguous(), 2, E)
    b.sync()
    Xa, Pa = a.indicator("X"), a.indicator("P")
    Xb, Pb = b.indicator("X"), b.indicator("P")
    # z is stored as given; x and y come back through the rotated angles
    # u = x + y, v = x - y, so only to their rounding
    assert np.array_equal(Xb[2], np.nextafter(Xa[2], np.inf))
    assert np.max(np.abs(Xb[:2] - Xa[:2])) < 4e-15
    assert np.array_equal(Pb[:2], Pa[:2])
    assert np.max(np.abs(Pb[2] - Pa[2])) < 1e-12
    assert np.max(np.abs(oracle.energy(1.0, Xb, Pb) - E)) < 1e-12
    a.close()
    b.close()


def test_diffusion_resume_rejects_an_inconsistent_checkpoint(tmp_path):
    """A checkpoint whose accumulated F does not hold the windows since the last
    snapshot boundary of the resumed schedule is refused, not silently used."""
    from paper_1107_4107_b300.experiments import diffusion_from_w
    kw = dict(n=1000, E=15.0, window_T=1.0, n_cos=8, n_phi=8, precision="fp32c")
    ck = str(tmp_path / "run.ckpt")
    diffusion_from_w(**kw, snapshots_T=(2.0,), ckpt_path=ck)     # stops at a boundary: F empty
    with pytest.raises(ValueError):
        diffusion_from_w(**kw, snapshots_T=(3.0,), ckpt_path=ck)   # would need windows 1-2 in F
    with open(ck, "r+b") as f:                                     # a truncated file
        f.truncate(100)
    with pytest.raises(Exception):
        diffusion_from_w(**kw, snapshots_T=(2.0, 4.0), ckpt_path=ck)


@pytest.mark.parametrize("precision", ["fp64", "df64f"])
def test_fig4_windows_match_oracle(precision):
    """Sec. IV, Fig. 4 on a small cloud: 500 trajectories Gaussian about W at
    E = 15, p_z from the energy with redraws, three windows of 1 T.  The kept
    initial conditions are exactly the draws the oracle's energy condition
    keeps (in order), and each time-averaged F of the runner equals the
    oracle's histogram of its own window velocities, up to bin-edge moves."""
    import oracle
    from paper_1107_4107_b300 import inputs
    from paper_1107_4107_b300.experiments import diffusion_from_w, init_gaussian_valid
    from parity import angle_dist, rel_err
    n, E, sigma, seed = 500, 15.0, 0.01, 0
    W = math.sqrt(E)
    h = 0.02 * math.pi
    w_steps = 100                                   # 1 T
    cand = max(2 * n, 1024)
    X, Pxy = inputs.gaussian_velocities(cand, (W, W), sigma, seed)
    P = np.zeros((3, cand))
    P[:2] = Pxy
    Po = oracle.pz_from_energy(E, 1.0, X, P)
    ok = np.isfinite(Po[2])
    assert 0.05 < ok.mean() < 0.95                  # the redraw really drops draws here
    Xk, Pk = X[:, ok][:, :n], Po[:, ok][:, :n]
    e = init_gaussian_valid(n, E, (W, W), sigma, seed, precision=precision, window=w_steps)
    assert np.max(angle_dist(e.indicator("X"), Xk)) < 1e-13
    assert rel_err(e.indicator("P"), Pk) < (1e-14 if precision == "fp64" else 1e-13)
    e.close()
    n_cos, n_phi = 16, 32
    run = diffusion_from_w(n=n, E=E, sigma=sigma, window_T=1.0, snapshots_T=(1.0, 3.0), n_cos=n_cos, n_phi=n_phi,
                           precision=precision, seed=seed)
    st = oracle.State(Xk, Pk, oracle.Params(h=h, window=w_steps), tangent=False)
    F = []
    for _ in range(3):
        st.advance(w_steps)
        F.append(oracle.velocity_histogram(st.velocity(), n_cos, n_phi))
    refs = [F[0], F[1] + F[2]]
    allowed = 2 if precision == "fp64" else 6
    for m, ref in zip(run["maps"], refs):
        got = m["counts"].astype(np.int64)
        assert got.sum() == ref.sum()
        assert np.abs(got - ref).sum() <= 2 * allowed, (m["t_T"], np.abs(got - ref).sum())
