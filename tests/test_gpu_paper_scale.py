"""The paper's own parameters (Section 3: E0 = 10^3.5, L = 10^1.5 in 2000
cells, dt = 10^-3.5, gamma_thr = 500, one particle per cell per species,
in-place pairs) against the FP64 oracle, for f = 0.1, 0.01 and 0.004.

The first photons are emitted at t_a = gamma_thr / E0 = 0.158 (step 500);
the runs go through two to four generations of pairs (1.1e6 particles at
step 1500 for f = 0.1, 0.8e6 and 2.0e6 at step 1000 for f = 0.01 and 0.004).
FP64: every per-step record and the E/J profiles to 1e-5 relative, every
count exact (the cold seed makes all particles of a species identical, so
nothing is chaotic yet).  FP32-mixed: the counts within 1% and the mean
field within 1e-3 of E0 at every step."""
import numpy as np
import pytest

import oracle
import test_gpu_parity as T
from paper_2012_05587_gb300 import Cascade, workloads as W

pytestmark = pytest.mark.gpu

CASES = [(0.1, 1500), (0.01, 1000), (0.004, 1000)]


@pytest.mark.parametrize("f,steps", CASES)
def test_fp64_per_step_parity(f, steps):
    p = W.paper_scale(f, "fp64")
    hz, r_ref, r_gpu = T.check_fp64_parity(p, steps, 100, min_horizon=steps + 1)
    assert r_ref["n_pairs_total"][-1] > 1e5  # the cascade has run several generations
    print(f"f = {f}: pairs {r_ref['n_pairs_total'][-1]}, particles {r_ref['n_elec'][-1] + r_ref['n_posi'][-1]}")


@pytest.mark.parametrize("f,steps", CASES)
def test_fp32_counts_and_field(f, steps):
    p = W.paper_scale(f, "fp32")
    d_ref = oracle.Oracle(T.oracle_params(p)).step(steps)
    with Cascade(p) as c:
        c.step(steps)
        d = c.diag(steps)
    for k in ("n_elec", "n_posi", "n_pairs_total"):
        assert abs(d[k][-1] - d_ref[k][-1]) <= 0.01 * d_ref[k][-1], k
    assert np.abs(d["E_mean"] - d_ref["E_mean"]).max() <= 1e-3 * p["E0"]
