"""Host-side helpers: the diagnostics analysis used in reports, the seeded
workloads, and the benchmark's reference-arm output contract."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2012_05587_gb300 import analysis as A, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_zero_crossings_of_a_sine():
    t = np.linspace(0.0, 10.0, 20001)
    z = A.zero_crossings(t, np.sin(2.0 * t + 0.3))
    want = (np.arange(1, 7) * np.pi - 0.3) / 2.0
    assert np.allclose(z, want[: len(z)], atol=1e-6)


def test_growth_rate_of_an_exponential_front():
    t = np.linspace(0.0, 5.0, 5001)
    n = np.minimum(10.0 * np.exp(3.0 * t), 1e6)
    assert A.growth_rate(t, n) == pytest.approx(3.0, rel=1e-3)


def test_closed_forms():
    # Eq. 3 for small f tends to ln(2/f); the renewal root tends to Eq. 3
    E0, g = 100.0, 1000.0
    ta = g / E0
    assert A.lambert_growth_rate(E0, g, 2.0) * ta == pytest.approx(np.log(1000.0) - np.log(np.log(1000.0)), rel=0.06)
    assert A.renewal_growth_rate(E0, g, 10.0) == pytest.approx(A.lambert_growth_rate(E0, g, 10.0), rel=0.03)
    assert A.mean_gamma(g, 10.0) == pytest.approx(g / np.log(200.0))
    assert A.screening_density(E0, g, 10.0) == pytest.approx(E0 * E0 * np.log(200.0) / (2 * g))


def test_ensemble_of_a_synthetic_record():
    t = np.linspace(0.01, 10.0, 1000)
    n = np.minimum(np.exp(2.0 * t), np.exp(2.0 * 4.0))
    rec = {"t": t, "E_mean": np.cos(3.0 * t) * np.exp(-0.01 * t), "n_elec": n, "n_posi": n,
           "n_pairs_total": n - 1, "U_E": t * 0, "U_K": t * 0 + 1, "U_gamma": t * 0}
    e = A.ensemble(rec)
    assert e["oscillation_frequency"] == pytest.approx(3.0, rel=1e-3)
    assert e["screening_time"] == pytest.approx(np.pi / 6.0, abs=0.02)
    assert e["growth_rate"] == pytest.approx(2.0, rel=0.02)


def test_batch_scan_is_seeded_and_bounded():
    a = W.batch_scan(32)
    b = W.batch_scan(32)
    assert a == b
    for p in a:
        assert 256 <= p["nx"] <= 8192 and p["ppc"] in (8, 16, 32, 64)
        assert 10 <= p["E0"] <= 1000 and p["eps_gamma"] >= 2 and p["gamma_thr"] - p["eps_gamma"] >= 1
        assert W.predicted_particles(p) <= (1 << 25)
        assert p["dt"] < p["dx"]


def test_corotating_state_satisfies_gauss_and_carries_j_m():
    p = W.corotating(nx=50, ppc=3)
    (c, o, u, q), E = W.corotating_state(p)
    w = p["n0"] * p["dx"] / p["ppc"]
    rho = np.bincount(c, weights=q.astype(float), minlength=p["nx"]) * w / p["dx"]
    assert np.allclose(rho, p["rho_gj"])
    v = u / np.sqrt(1 + u * u)
    J = (q * v).sum() * w / (p["nx"] * p["dx"])
    assert J == pytest.approx(p["j_m"])
    assert np.all(E == 0)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "1", "--prep", "10"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "particle-steps/s" and line["value"] > 0
    assert line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_damping_rate_of_a_damped_oscillation():
    """Eq. 24's envelope: a cosine whose amplitude holds for 5 time units and
    then decays as exp(-0.08 t); the fit over the peaks between 0.9 and 0.4
    of the first peak recovers the rate, and an undamped cosine gives zero."""
    t = np.linspace(0.0, 60.0, 60001)
    env = np.where(t < 5.0, 1.0, np.exp(-0.08 * (t - 5.0)))
    lam, n = A.damping_rate(t, 40.0 * env * np.cos(3.0 * t + 0.2))
    assert lam == pytest.approx(0.08, rel=0.02) and n >= 5
    lam0, _ = A.damping_rate(t, 40.0 * np.cos(3.0 * t + 0.2))
    assert abs(lam0) < 1e-4


def test_growth_rate_between_counts():
    """The rate between two fixed counts of an exponential, whatever the
    sampling, and the window of the parameters (Eq. 5 multiplicity)."""
    t = np.linspace(0.0, 3.0, 301)
    n = 1000.0 * np.exp(2.5 * t)
    assert A.growth_rate_between(t, n, 4000.0, 400000.0) == pytest.approx(2.5, rel=1e-4)
    p = dict(nx=256, ppc=4, n0=1.0, E0=100.0, gamma_thr=50.0, eps_gamma=5.0)
    lo, hi = A.growth_window(p)
    n_seed = 2 * 256 * 4
    assert lo == 4 * n_seed and hi == pytest.approx(n_seed * A.screening_density(100.0, 50.0, 5.0) / 4)
    assert A.growth_window(dict(p, E0=10.0, gamma_thr=20.0, eps_gamma=10.0)) is None  # one generation only
    # the seed average of ln N: two runs growing at 2.0 and 3.0 with the same
    # start average to 2.5 between the counts
    recs = [{"t": t, "n_elec": 500.0 * np.exp(r * t), "n_posi": 500.0 * np.exp(r * t)} for r in (2.0, 3.0)]
    assert A.seed_averaged_growth_rate(recs, (4000.0, 400000.0)) == pytest.approx(2.5, rel=1e-3)


def test_paired_comparison_reports_bias_and_its_error():
    rng = np.random.default_rng(0)
    base = rng.normal(1.0, 0.2, 400)
    refs = [{"x": v, "seed": i} for i, v in enumerate(base)]
    runs = [{"x": v * 1.03 + rng.normal(0.0, 0.01), "seed": i} for i, v in enumerate(base)]
    c = A.paired_comparison(runs, refs)["x"]
    assert c["rel_err"] == pytest.approx(0.03, abs=0.003)
    assert 0.0 < c["rel_se"] < 0.002 and c["n"] == 400


def test_stratified_sample_sizes():
    import bench_workloads as BW

    items = list(range(10))
    assert BW.stratified(items, 0, lambda x: x) == []
    assert BW.stratified(items, -1, lambda x: x) == items
    assert BW.stratified(items, 20, lambda x: x) == items
    got = BW.stratified(items, 5, lambda x: -x)  # sorted by key, spread evenly
    assert len(got) == 5 and len(set(got)) == 5
    assert got == [8, 6, 4, 2, 0]  # the middle of each fifth of [9, 8, ..., 0]
