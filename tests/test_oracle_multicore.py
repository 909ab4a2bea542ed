"""The multi-core (OpenMP) build of the oracle, used only to time the CPU on
all host cores, against the plain build: bit-identical on one thread, and on
several threads equal counts with round-off differences in the sums of the
charge-conserving deposit and the diagnostics (Section 3 small cascade)."""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import workloads as W


@pytest.fixture(scope="module")
def mc_lib():
    try:
        return oracle.build_multicore()
    except Exception as e:  # pragma: no cover - compiler without OpenMP
        pytest.skip(f"no OpenMP build: {e}")


def small():
    p = {k: v for k, v in W.small_cascade().items() if k != "precision"}
    return p


def run(p, lib, threads, steps):
    oracle._load(lib).orc_set_threads(threads)
    o = oracle.Oracle(p, lib_path=lib)
    d = o.step(steps)
    E, J = o.fields()
    return d, E, J


def test_one_thread_is_bit_identical(mc_lib):
    p = small()
    d0, E0, J0 = run(p, None, 1, 300)
    d1, E1, J1 = run(p, mc_lib, 1, 300)
    assert oracle._load(mc_lib).orc_threads() == 1
    for f in d0:
        assert np.array_equal(d0[f], d1[f]), f
    assert np.array_equal(E0, E1) and np.array_equal(J0, J1)


def test_four_threads_match_to_round_off(mc_lib):
    p = small()
    d0, E0, J0 = run(p, None, 1, 300)
    d4, E4, J4 = run(p, mc_lib, 4, 300)
    assert oracle._load(mc_lib).orc_threads() == 4
    assert d0["n_pairs_total"][-1] > 0
    for f in ("n_elec", "n_posi", "n_photon", "n_pairs_total"):
        assert np.array_equal(d0[f], d4[f]), f
    scale = np.abs(d0["E_absmax"]).max()
    assert np.abs(d4["E_mean"] - d0["E_mean"]).max() <= 1e-9 * scale
    assert np.abs(E4 - E0).max() <= 1e-9 * scale
    assert np.allclose(d4["U_K"], d0["U_K"], rtol=1e-12)
    assert np.abs(d4["gauss_resid"]).max() <= 1e-10 * scale
