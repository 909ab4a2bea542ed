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
