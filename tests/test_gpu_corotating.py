"""Co-rotating frame (Section 7, Eq. 25-26) and open boundaries on the GPU,
against the oracle through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import Cascade, CascadeError, capi, workloads as W

import test_gpu_parity as T
from test_oracle_corotating import cold_state

pytestmark = pytest.mark.gpu


def split(c, o, u, q):
    e, p = q < 0, q > 0
    return ({"cell": c[e], "off": o[e], "u": u[e]}, {"cell": c[p], "off": o[p], "u": u[p]})


def run_pair(p, state, E, steps, chunk=50):
    c, o, u, q = state
    ref = oracle.Oracle.from_state(T.oracle_params(p), c, o, u, q, E=E)
    elec, posi = split(c, o, u, q)
    recs, rrecs, snaps = [], [], []
    with Cascade(p, state={"elec": elec, "posi": posi, "E": E}) as g:
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            rrecs.append(ref.step(k))
            g.step(k)
            recs.append(g.diag(k))
            Eg, Jg = g.fields()
            Er, Jr = ref.fields()
            done += k
            snaps.append((done, Eg, Jg, Er, Jr, g.gauss()))
    cat = lambda rs: {f: np.concatenate([r[f] for r in rs]) for f in rs[0]}
    return cat(rrecs), cat(recs), snaps


def base(**kw):
    p = dict(nx=64, ppc=4, dx=0.1, dt=0.02, n0=1.0, u_spread=0.0, seed=1, E0=0.0, gamma_thr=1e9,
             eps_gamma=10.0, l_pp=0.0, j_m=0.0, rho_gj=0.0, open_bc=0, particle_cap=1 << 16, precision="fp64")
    p.update(kw)
    return p


def test_corotating_equilibrium_stays_put():
    v = 0.5
    uu = v / np.sqrt(1 - v * v)
    p = base(nx=16, dt=0.01, j_m=1.5, rho_gj=-1.0)
    state = cold_state(16, 8, 4, -uu, uu)
    r_ref, r_gpu, snaps = run_pair(p, state, np.zeros(16), 1000, chunk=250)
    assert np.abs(r_gpu["E_absmax"]).max() <= 1e-10
    for _, Eg, _, _, _, gres in snaps:
        assert gres <= 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_open_outflow_matches_oracle(precision, tol):
    """A positron beam with its self-consistent field streams out through
    x = L: counts exactly, E and J per step, Gauss on interior nodes."""
    nx, dx = 64, 0.1
    p = base(nx=nx, dx=dx, open_bc=1, precision=precision)
    state = cold_state(nx, 0, 4, 0.0, 0.8)
    E = (np.arange(nx) + 0.5) * dx
    r_ref, r_gpu, snaps = run_pair(p, state, E, 600)
    E_scale = np.abs(E).max()  # the field decays to ~0 once the beam has left
    if precision == "fp64":
        assert np.array_equal(r_gpu["n_posi"], r_ref["n_posi"])
    else:
        assert np.abs(r_gpu["n_posi"] - r_ref["n_posi"]).max() <= 2
    assert r_gpu["n_posi"][-1] < r_gpu["n_posi"][0] / 2
    for _, Eg, Jg, Er, Jr, gres in snaps:
        assert np.abs(Eg - Er).max() <= tol * E_scale
        assert gres <= (1e-12 if precision == "fp64" else 1e-4) * E_scale


def test_departures_and_dropped_photons_are_exact():
    """Single particles crossing x = L and x = 0 leave in the same step as in
    the oracle; a photon that would convert outside is not kept."""
    p = base(nx=20, dx=0.1, dt=0.01, n0=1e-12, open_bc=1, particle_cap=64)
    u = 3.0
    state = (np.array([19, 0]), np.array([0.5, 0.5]), np.array([u, -u]), np.array([1, -1]))
    r_ref, r_gpu, _ = run_pair(p, state, np.zeros(20), 30, chunk=30)
    assert np.array_equal(r_gpu["n_posi"], r_ref["n_posi"]) and np.array_equal(r_gpu["n_elec"], r_ref["n_elec"])
    assert r_gpu["n_posi"][-1] == 0 and r_gpu["n_elec"][-1] == 0
    q = base(nx=20, dx=0.1, dt=0.01, n0=1e-14, E0=1.0, gamma_thr=20.0, eps_gamma=4.0, l_pp=0.55, open_bc=1,
             particle_cap=64)
    for u0, E in ((19.99, np.full(20, 1.0)), (-19.99, np.full(20, -1.0))):
        st = (np.array([19]), np.array([0.2]), np.array([u0]), np.array([1]))
        r_ref, r_gpu, _ = run_pair(q, st, E, 1, chunk=1)
        assert r_gpu["n_photon"][0] == r_ref["n_photon"][0]
        assert r_gpu["U_K"][0] == pytest.approx(r_ref["U_K"][0], rel=1e-12)


def test_small_corotating_discharge_matches_oracle():
    """A scaled-down Section 7 run: the cold two-density state with j_m, open
    boundaries and pair creation; per-step parity to the horizon (FP64)."""
    p = W.corotating(nx=400, precision="fp64", gamma_thr=60.0, eps_gamma=6.0, dt=0.02)
    state, E = W.corotating_state(p)
    steps = 1500
    r_ref, r_gpu, snaps = run_pair(p, state, E, steps, chunk=100)
    hz = T.horizon(r_ref, r_gpu)
    assert r_ref["n_pairs_total"][-1] > 0
    assert hz >= 200
    m = r_ref["step"] < hz
    scale = np.abs(r_ref["E_absmax"][m]).max()
    assert np.abs(r_gpu["E_mean"][m] - r_ref["E_mean"][m]).max() <= T.RTOL * scale
    for done, Eg, _, Er, _, gres in snaps:
        assert gres <= 1e-10 * max(1.0, np.abs(Er).max())
        if done < hz:
            assert np.abs(Eg - Er).max() <= T.RTOL * max(np.abs(Er).max(), 1e-12)


def test_open_boundaries_rejected_in_batches():
    p = base(open_bc=1, precision="fp32")
    from paper_2012_05587_gb300 import CascadeBatch

    with CascadeBatch(slots=2, precision="fp32", max_nx=128) as b:
        with pytest.raises(CascadeError) as ei:
            b.admit(p, 10)
        assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG


def test_open_boundaries_on_a_grid_beyond_shared_memory():
    """Nx = 40000 in FP32: E does not fit beside the accumulator, so the open-
    boundary particle kernel reads E through L1.  The Section 7 state (j_m,
    rho_GJ, open ends), 100 steps against the oracle: E per edge, the interior
    Gauss residual and the species counts."""
    p = W.corotating(nx=40000, precision="fp32", gamma_thr=60.0, eps_gamma=6.0, dt=0.02)
    state, E = W.corotating_state(p)
    r_ref, r_gpu, snaps = run_pair(p, state, E, 100, chunk=100)
    done, Eg, _, Er, _, gres = snaps[-1]
    scale = max(np.abs(Er).max(), 1e-12)
    assert np.abs(Eg - Er).max() <= 2e-4 * scale
    assert gres <= 1e-4 * max(1.0, scale)
    for k in ("n_elec", "n_posi"):
        assert np.abs(r_gpu[k] - r_ref[k]).max() <= 2
