"""Edge cases of the CUDA path against the oracle through the C ABI: grids
too large for shared memory (the particle kernel then reads E, or also adds
the current, through global memory), and a state with no particles at all
(the degenerate case: Ampere with J = 0 and a background current only)."""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import Cascade

import test_gpu_parity as T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,nx,ppc,tol", [
    ("fp32", 40000, 1, 2e-4),   # E (160 KB) and the accumulator do not fit together: E read through L1
    ("fp32", 60000, 1, 2e-4),   # neither fits: E and the current both in global memory
    ("fp64", 30000, 1, 1e-9),   # FP64 E does not fit: global E and FP64 global atomics
])
def test_grids_beyond_shared_memory_match_oracle(precision, nx, ppc, tol):
    """The large cascade's physics (E0 = 100, gamma_thr = 50, eps = 20, l_pp =
    0.5, dt = 0.025, dx = 0.05) on grids that leave the shared-memory layout,
    60 steps through the first emissions and conversions: E and J per edge
    and the pair count against the FP64 oracle."""
    from paper_2012_05587_gb300 import workloads as W

    p = dict(W.large_cascade(precision=precision), nx=nx, ppc=ppc, particle_cap=1 << 20)
    steps = 60
    ref = oracle.Oracle(T.oracle_params(p))
    d_ref = ref.step(steps)
    E_ref, J_ref = ref.fields()
    with Cascade(p) as c:
        c.step(steps)
        d = c.diag(steps)
        E, J = c.fields()
    assert d_ref["n_pairs_total"][-1] > 0
    assert np.abs(E - E_ref).max() <= tol * np.abs(E_ref).max()
    assert np.abs(J - J_ref).max() <= 10 * tol * np.abs(J_ref).max()
    assert abs(d["n_pairs_total"][-1] - d_ref["n_pairs_total"][-1]) <= 0.01 * d_ref["n_pairs_total"][-1]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_empty_state_follows_the_background_current(precision):
    """No particles: J = 0, so Ampere with a background current j_m gives
    E^n = E^0 + n dt j_m exactly (Eq. 26); counts stay zero, U_K = 0."""
    nx, dt, jm = 64, 0.01, 0.25
    p = dict(nx=nx, ppc=1, dx=0.1, dt=dt, n0=1.0, u_spread=0.0, seed=1, E0=0.0, gamma_thr=50.0, eps_gamma=10.0,
             l_pp=0.0, j_m=jm, particle_cap=1024, precision=precision)
    empty = {"cell": np.zeros(0, np.int32), "off": np.zeros(0), "u": np.zeros(0)}
    E0 = np.linspace(-1.0, 1.0, nx)
    steps = 200
    ref = oracle.Oracle.from_state(T.oracle_params(p), [], [], [], [], E=E0)
    d_ref = ref.step(steps)
    E_ref, _ = ref.fields()
    with Cascade(p, state={"elec": empty, "posi": empty, "E": E0}) as c:
        c.step(steps)
        d = c.diag(steps)
        E, J = c.fields()
    assert np.all(d["n_elec"] == 0) and np.all(d["n_posi"] == 0) and np.all(d["n_pairs_total"] == 0)
    assert np.all(d["U_K"] == 0.0)
    assert np.all(J == 0.0)
    assert np.allclose(E, E0 + steps * dt * jm, rtol=0, atol=1e-12)
    assert np.array_equal(E, E_ref)
    assert np.allclose(d["E_mean"], d_ref["E_mean"], rtol=0, atol=1e-13)


def test_photon_ring_overflow_is_reported():
    """A photon ring smaller than one step's emissions: the photons that do not
    fit are dropped and the run reports CASCADE_ERR_PHOTON_CAPACITY (the ring
    index is checked before every append)."""
    from paper_2012_05587_gb300 import CascadeError, capi, workloads as W

    p = dict(W.small_cascade(), photon_cap=64)
    with Cascade(p) as c:
        c.step(120)  # the seed reaches gamma_thr after t_a = 2 (40 steps); 8192 leptons emit together
        with pytest.raises(CascadeError) as ei:
            c.sync()
        assert ei.value.status == capi.CASCADE_ERR_PHOTON_CAPACITY


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_runaway_energy_is_reported(precision):
    """A field so strong that one push takes u past 1e30: the particle kernel
    flags CASCADE_ERR_NONFINITE instead of emitting from a meaningless gamma."""
    from paper_2012_05587_gb300 import CascadeError, capi, workloads as W

    p = dict(W.small_cascade(precision=precision), E0=1e33)
    with Cascade(p) as c:
        c.step(3)
        with pytest.raises(CascadeError) as ei:
            c.sync()
        assert ei.value.status == capi.CASCADE_ERR_NONFINITE
