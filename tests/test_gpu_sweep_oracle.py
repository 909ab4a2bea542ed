"""The precision sweep's cascading rows in FP32 against the FP64 oracle.

Rows (E0, gamma_thr) = (10, 20), (100, 20), (100, 200), (1000, 2000) of the
precision sweep (Nx = 4096, 32 + 32 per cell, eps = gamma_thr / 2, l_pp = 1,
5000 steps) run on an Nx = 512 slice -- the same dx, dt, seed density,
seeds and physics -- because the oracle cannot run the full grid in a test.
The oracle's ensemble diagnostics of the 8 seeds of each row are stored in
tests/golden/sweep_oracle.json, written by tests/golden/make_sweep_oracle.py
(which runs the oracle only).  Here FP32-mixed runs the same slices and
seeds on the GPU.  Diagnostics that the cascade fixes (growth rate,
screening time, peak field after screening, plateau frequency, final
energy) must agree to 2%; those that the instability of Section 5 decides
after the parity horizon (the damping rate, the pair count after the
secondary bursts) to 2% up to three standard errors of the seed-by-seed
differences.  The damping rate is compared through the decay of the
envelope over the run, D = rate x (steps dt): relatively (2%) where the
oracle's envelope falls by at least a factor e, absolutely (0.02) where it
barely decays and the rate is near zero.  The test prints every error."""
import json
import os

import numpy as np
import pytest

from paper_2012_05587_gb300 import Cascade, analysis as A, workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sweep_oracle.json")
TOL = 0.02
FIXED = ("growth_rate", "screening_time", "peak_field_after_screening", "oscillation_frequency", "final_energy")
CHAOTIC = ("final_pairs",)


def _gold():
    with open(GOLD) as f:
        return json.load(f)


@pytest.mark.parametrize("row", [0, 3, 4, 8])
def test_fp32_sweep_row_against_the_oracle(row):
    gold = _gold()
    entry = next(r for r in gold["rows"] if r["row"] == row)
    refs = entry["diagnostics"]
    runs = []
    for run in range(len(refs)):
        p = W.precision_sweep(run=run, precision="fp32")[row]
        p = {k: v for k, v in p.items() if k != "steps"}
        p.update(nx=gold["nx"], particle_cap=1 << 26)
        assert p["seed"] == refs[run]["seed"]
        with Cascade(p) as c:
            c.step(gold["steps"])
            runs.append(A.ensemble(c.diag(gold["steps"]), p))
    cmp = A.paired_comparison(runs, refs, FIXED + CHAOTIC)
    for k, v in cmp.items():
        print(f"row {row} {k:28s} fp32 {v['mean']:.6g} oracle {v['ref_mean']:.6g} "
              f"rel {v['rel_err']:+.4f} +- {v['rel_se']:.4f}")
    for k in FIXED:
        if np.isfinite(cmp[k]["ref_mean"]):
            assert abs(cmp[k]["rel_err"]) <= TOL, k
    for k in CHAOTIC:
        if np.isfinite(cmp[k]["rel_err"]):
            assert abs(cmp[k]["rel_err"]) <= TOL + 3 * cmp[k]["rel_se"], k
    # damping: the envelope's decay over the run
    T = gold["steps"] * entry["dt"]
    D = np.array([r["damping_rate"] for r in runs]) * T
    D_ref = np.array([r["damping_rate"] for r in refs]) * T
    diff = D - D_ref
    se = diff.std(ddof=1) / np.sqrt(len(diff))
    print(f"row {row} damping decay over the run: fp32 {D.mean():.4f} oracle {D_ref.mean():.4f} "
          f"diff {diff.mean():+.4f} +- {se:.4f}")
    if D_ref.mean() >= 1.0:
        assert abs(diff.mean()) <= TOL * D_ref.mean() + 3 * se
    else:
        assert abs(diff.mean()) <= TOL + 3 * se
