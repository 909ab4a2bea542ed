"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed-form solutions of special cases of the same
equations, conservation laws, and the analytic results of arXiv:2012.05587
(Sections 3-5).  ``test_oracle_mutants.py`` shows that plausible mistakes in the
oracle fail these pins.
"""
import os

import numpy as np
import pytest

import fitting as F
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def base_params(**kw):
    p = dict(nx=8, ppc=4, dx=0.1, dt=0.01, n0=1.0, u_spread=0.0, seed=1, E0=1e-4,
             gamma_thr=1e9, eps_gamma=10.0, l_pp=0.0)
    p.update(kw)
    return p


def quiet_positions(nx, ppc):
    i = np.repeat(np.arange(nx), ppc)
    k = np.tile(np.arange(ppc), nx)
    return i, (k + 0.5) / ppc


# --- random numbers -----------------------------------------------------------

def test_philox_known_answers(lib=None):
    """Philox4x32-10 against the published known-answer vectors (Salmon et al. 2011)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6], lib)
        assert list(out) == v[6:10]


def test_seed_normals_are_standard_normal(lib=None):
    z = np.array([oracle.seed_normals(1234, j, lib) for j in range(40000)]).ravel()
    assert abs(z.mean()) < 4.0 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 6.0 * np.sqrt(2.0 / len(z))
    # tails of a normal: P(|z| > 2) = 0.0455
    assert abs(np.mean(np.abs(z) > 2.0) - 0.0455) < 0.004
    # independence of the two Box-Muller branches
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.02


# --- initial condition ----------------------------------------------------------

def test_quiet_start_layout_and_gauss(lib=None):
    p = base_params(nx=16, ppc=8, u_spread=0.01, seed=99, E0=3.0)
    o = oracle.Oracle(p, lib)
    st = o.particles()
    assert o.num_particles == 2 * 16 * 8
    # pair j: electron then positron, cell j mod nx, offset (j div nx + 1/2) / ppc
    j = np.arange(16 * 8)
    assert np.array_equal(st["cell"][0::2], j % 16) and np.array_equal(st["cell"][1::2], j % 16)
    assert np.allclose(st["off"][0::2], (j // 16 + 0.5) / 8, rtol=0, atol=0)
    assert np.all(st["q"][0::2] == -1) and np.all(st["q"][1::2] == 1)
    ze, zp = oracle.seed_normals(99, 5, lib)
    assert st["u"][10] == 0.01 * ze and st["u"][11] == 0.01 * zp
    d = o.diag_now()
    assert d["gauss_resid"] == 0.0 and d["E_mean"] == 3.0
    assert d["n_elec"] == d["n_posi"] == 128


# --- push and move ------------------------------------------------------------

def _single_particle_error(dt, T=10.0, E0=1.0, u0=0.3, lib=None):
    p = base_params(nx=4096, ppc=1, dx=0.1, dt=dt, n0=1e-14, E0=E0)
    c0, o0 = 100, 0.5
    orc = oracle.Oracle.from_state(p, [c0], [o0], [u0], [1], lib_path=lib)
    n = int(round(T / dt))
    orc.step(n)
    st = orc.particles()
    # u^{n-1/2} after n pushes in the frozen uniform field: u0 + q E0 n dt
    assert st["u"][0] == pytest.approx(u0 + E0 * n * dt, rel=1e-13)
    # leapfrog u is staggered by dt/2: u(t) = u0 + E0 (t + dt/2); x(t) from energy
    ua = u0 + E0 * 0.5 * dt
    ub = u0 + E0 * (n * dt + 0.5 * dt)
    x_exact = (c0 + o0) * 0.1 + (np.sqrt(1 + ub * ub) - np.sqrt(1 + ua * ua)) / E0
    x_num = (st["cell"][0] + st["off"][0]) * 0.1
    return x_num - x_exact


def test_single_particle_uniform_field_second_order(lib=None):
    e1 = _single_particle_error(0.02, lib=lib)
    e2 = _single_particle_error(0.01, lib=lib)
    assert abs(e1) < 1e-4
    assert 3.5 < abs(e1 / e2) < 4.5


def test_electron_moves_against_field(lib=None):
    p = base_params(nx=64, ppc=1, dx=0.1, dt=0.01, n0=1e-14, E0=2.0)
    orc = oracle.Oracle.from_state(p, [32], [0.5], [0.0], [-1], lib_path=lib)
    orc.step(50)
    st = orc.particles()
    assert st["u"][0] == pytest.approx(-2.0 * 50 * 0.01, rel=1e-13)
    assert (st["cell"][0] + st["off"][0]) < 32.5


# --- deposit + Ampere -------------------------------------------------------------

def test_gauss_and_charge_conservation_with_qed(lib=None):
    """Charge-conserving deposit: Gauss's law stays at round-off while pairs
    are created (pairs are born co-located, so rho is unchanged)."""
    p = dict(nx=64, ppc=8, dx=0.1, dt=0.05, n0=1.0, u_spread=0.01, seed=4321, E0=10.0,
             gamma_thr=20.0, eps_gamma=10.0, l_pp=1.0, particle_cap=100000)
    o = oracle.Oracle(p, lib)
    d = o.step(1500)
    assert d["n_pairs_total"][-1] > 0
    assert np.all(d["gauss_resid"] <= 1e-12 * np.maximum(d["E_absmax"], 1.0))
    assert np.array_equal(d["n_elec"], d["n_posi"])


def test_mean_current_and_field_of_a_hand_built_state(lib=None):
    """The per-step field diagnostics on a state whose values are fixed by
    definitions outside the oracle: two charges moving at known speed in a
    region where the field is zero (so they are not pushed), one of them
    crossing a node.

    * <J> is the domain average of the current density of the moving
      macro-particles, sum over particles of q w v / L (w = n0 dx / ppc per
      unit area, L = nx dx), whatever the deposit stencil;
    * <E> then follows from Ampere's law averaged over the periodic domain,
      <E>^{n+1} = <E>^n - dt <J>;
    * max |E| is attained at an edge other than 0 and by a negative value."""
    p = dict(nx=8, ppc=1, dx=0.1, dt=0.01, n0=1.0, u_spread=0.0, seed=1, E0=0.0,
             gamma_thr=1e9, eps_gamma=10.0, l_pp=0.0)
    E = np.array([1.0, -5.0, 0.0, 0.0, 3.5, 0.0, 0.0, 2.0])
    # a positron at v = +0.6 (u = 3/4) and an electron at v = -0.8 (u = -4/3)
    # that crosses the node at x = 6 dx; both sit between edges where E = 0
    u = np.array([0.75, -4.0 / 3.0])
    q = np.array([1, -1])
    o = oracle.Oracle.from_state(p, [3, 6], [0.2, 0.03], u, q, E=E, lib_path=lib)
    d = o.step(1)
    w, L = p["n0"] * p["dx"] / p["ppc"], p["nx"] * p["dx"]
    v = u / np.sqrt(1.0 + u * u)
    J_mean = float((q * w * v).sum() / L)
    assert J_mean == pytest.approx(0.175, rel=1e-15)
    assert d["J_mean"][0] == pytest.approx(J_mean, rel=1e-12)
    assert d["E_mean"][0] == pytest.approx(E.mean() - p["dt"] * J_mean, rel=1e-12)
    assert d["E_absmax"][0] == pytest.approx(5.0, rel=1e-15)
    st = o.particles()
    assert np.array_equal(st["cell"], [3, 5])  # the electron crossed into cell 5


def test_cold_uniform_mode_frequency(lib=None):
    """Linear cold uniform mode of a pair plasma: 2 sin(w dt/2)/dt = sqrt(2 n0)."""
    dt = 0.01
    o = oracle.Oracle(base_params(dt=dt), lib)
    d = o.step(22000)
    w = 2 * np.pi / F.period_from_crossings(d["t"], d["E_mean"])
    assert w == pytest.approx(F.leapfrog_uniform_mode_omega(1.0, dt), rel=1e-6)


def test_relativistic_uniform_mode_period(lib=None):
    """Cold uniform mode from u = 0 in E0 = 2: period from the energy integral,
    reached at second order in dt."""
    Tq = F.relativistic_uniform_mode_period(2.0, 1.0)
    errs = []
    for dt in (0.004, 0.002):
        o = oracle.Oracle(base_params(E0=2.0, dt=dt), lib)
        d = o.step(int(6 * Tq / dt))
        errs.append(F.period_from_crossings(d["t"], d["E_mean"]) / Tq - 1.0)
    assert abs(errs[1]) < 1e-6
    assert 3.0 < errs[0] / errs[1] < 5.0


def _standing_wave(dt, mutant=None):
    nx, ppc, dx = 64, 32, 0.1
    k = 2 * np.pi / (nx * dx)
    i, off = quiet_positions(nx, ppc)
    x = (i + off) * dx
    a = 1e-3
    p = base_params(nx=nx, ppc=ppc, dx=dx, dt=dt, E0=0.0)
    cell = np.concatenate([i, i])
    offs = np.concatenate([off, off])
    u = np.concatenate([-a * np.sin(k * x), a * np.sin(k * x)])
    q = np.concatenate([-np.ones(len(i)), np.ones(len(i))])
    o = oracle.Oracle.from_state(p, cell, offs, u, q, lib_path=mutant)
    return o.step(int(40 / dt))


def test_standing_langmuir_wave(lib=None):
    """k != 0 Langmuir wave in a cold pair plasma: frequency sqrt(2 n0) up to the
    O((k dx)^2) grid correction, and no secular energy drift (field energy and
    kinetic energy trade exactly through the matched gather and deposit)."""
    dt = 0.01
    d = _standing_wave(dt, lib)
    ue = d["U_E"] - d["U_E"].mean()
    w = np.pi / F.period_from_crossings(d["t"], ue)
    assert w == pytest.approx(F.leapfrog_uniform_mode_omega(1.0, dt), rel=2e-3)
    tot = d["U_E"] + d["U_K"]
    per = int(round(np.pi / w / dt))
    drift = abs(tot[-2 * per:].mean() - tot[:2 * per].mean())
    assert drift < 1e-3 * d["U_E"].max()
    assert d["gauss_resid"].max() < 1e-14


def test_energy_conservation_with_cascade(lib=None):
    """Total energy U_E + U_K + U_gamma: emission and conversion conserve it
    exactly; the PIC scheme to first order in dt for this half-step kinetic
    energy."""
    dev = []
    for dt in (0.05, 0.025):
        p = dict(nx=128, ppc=16, dx=0.1, dt=dt, n0=1.0, u_spread=0.01, seed=2234, E0=10.0,
                 gamma_thr=20.0, eps_gamma=10.0, l_pp=1.0, particle_cap=100000)
        d = oracle.Oracle(p, lib).step(int(20 / dt))
        tot = d["U_E"] + d["U_K"] + d["U_gamma"]
        t0 = 0.5 * 10.0 ** 2 * 128 * 0.1 + 2 * 128 * 16 * (0.1 / 16) * np.sqrt(1.0)
        assert abs(tot[-1] - t0) / t0 < 1e-3
        dev.append(np.abs(tot - t0).max() / t0)
        assert d["n_pairs_total"][-1] > 0
    assert dev[0] < 1e-2
    assert dev[1] < 0.6 * dev[0]


# --- QED model ------------------------------------------------------------------

def _frozen(**kw):
    p = base_params(nx=400, ppc=1, dx=0.1, dt=0.01, n0=1e-14, E0=10.0, gamma_thr=20.0,
                    eps_gamma=4.0, l_pp=0.55, particle_cap=1000)
    p.update(kw)
    return p


def test_single_emission_bookkeeping(lib=None):
    """A positron accelerated through gamma_thr emits one photon, recoils by
    eps_gamma keeping its direction, and the photon becomes an e-/e+ pair of
    gamma = eps_gamma / 2 each, n_pp steps later, l_pp further along (Section 2)."""
    p = _frozen(E0=1.0)  # slow enough that the recoiled positron stays below threshold
    u0 = 19.0
    o = oracle.Oracle.from_state(p, [50], [0.3], [u0], [1], lib_path=lib)
    npp = o.n_pp
    assert npp == 55
    # first step with gamma >= 20: u0 + n * 0.01 >= sqrt(399)
    n_emit = int(np.ceil((np.sqrt(20.0 ** 2 - 1) - u0) / (1.0 * 0.01)))
    d = o.step(n_emit - 1)
    assert d["n_photon"][-1] == 0
    d = o.step(1)
    assert d["n_photon"][-1] == 1 and d["n_pairs_total"][-1] == 0
    st = o.particles()
    ph = o.photons()
    g_after = np.sqrt(1 + st["u"][0] ** 2)
    g_before = np.sqrt(1 + (u0 + n_emit * 0.01) ** 2)
    assert g_after == pytest.approx(g_before - 4.0, rel=1e-14)
    assert st["u"][0] > 0
    x_emit = st["cell"][0] + st["off"][0]
    assert ph["dir"][0] == 1
    assert ph["conv_step"][0] == n_emit + npp
    assert ph["cell"][0] + ph["off"][0] == pytest.approx(x_emit + 0.55 / 0.1, abs=1e-12)
    w = p["n0"] * p["dx"] / p["ppc"]
    assert d["U_gamma"][-1] == pytest.approx(w * 4.0, rel=1e-15)
    # emitted at t = n_emit dt; converts at t = (n_emit + n_pp) dt, i.e. at the
    # start of the step after the next n_pp ones
    d = o.step(npp)
    assert d["n_pairs_total"][-1] == 0 and d["n_photon"][-1] == 1
    d = o.step(1)
    assert d["n_pairs_total"][-1] == 1 and d["n_photon"][-1] == 0
    assert d["n_elec"][-1] == 1 and d["n_posi"][-1] == 2
    st = o.particles()
    # the new pair sat at the conversion point with gamma = eps/2 before this push
    up = np.sqrt(2.0 ** 2 - 1)
    assert st["u"][1] == pytest.approx(up - 1.0 * 0.01, rel=1e-13)  # electron decelerated
    assert st["u"][2] == pytest.approx(up + 1.0 * 0.01, rel=1e-13)  # positron accelerated


def test_electron_emission_runs_backwards(lib=None):
    p = _frozen(l_pp=0.3)
    o = oracle.Oracle.from_state(p, [200], [0.7], [-19.95], [-1], lib_path=lib)
    d = o.step(1)
    assert d["n_photon"][-1] == 1
    st, ph = o.particles(), o.photons()
    assert ph["dir"][0] == -1 and st["u"][0] < 0
    assert ph["cell"][0] + ph["off"][0] == pytest.approx(st["cell"][0] + st["off"][0] - 3.0, abs=1e-12)


def test_multi_photon_emission_conserves_energy(lib=None):
    """gamma far above threshold: k = 1 + floor((gamma - gamma_thr)/eps) photons."""
    p = _frozen(l_pp=0.0)
    u0 = 31.0
    o = oracle.Oracle.from_state(p, [10], [0.5], [u0], [1], lib_path=lib)
    before = o.diag_now()
    d = o.step(1)
    g = np.sqrt(1 + (u0 + 0.1) ** 2)
    k = 1 + int(np.floor((g - 20.0) / 4.0))
    assert k == 3
    assert d["n_photon"][0] == k and d["n_emit_multi"][0] == 1
    w = p["n0"] * p["dx"]
    # kinetic + photon energy after the step = kinetic energy after the push
    assert d["U_K"][0] + d["U_gamma"][0] == pytest.approx(w * g, rel=1e-14)
    assert before["U_gamma"] == 0.0
    d = o.step(1)  # l_pp = 0: converted at the start of the next step
    assert d["n_pairs_total"][0] == 3 and d["n_photon"][0] == 0


def test_threshold_tie_emits(lib=None):
    """gamma exactly at gamma_thr emits (a lepton that reaches gamma_thr)."""
    p = _frozen(E0=0.0, n0=1e-14)
    u_thr = np.sqrt(20.0 ** 2 - 1.0)
    assert np.sqrt(1.0 + u_thr * u_thr) >= 20.0
    o = oracle.Oracle.from_state(p, [10], [0.5], [u_thr], [1], lib_path=lib)
    d = o.step(1)
    assert d["n_photon"][0] == 1


def test_in_place_conversion(lib=None):
    """l_pp = 0 is the paper's in-place conversion: a photon emitted at step n
    converts before the push of step n+1, at the emitter's position."""
    p = _frozen(l_pp=0.0)
    o = oracle.Oracle.from_state(p, [10], [0.5], [19.9], [1], lib_path=lib)
    assert o.n_pp == 0
    d = o.step(1)
    assert d["n_photon"][0] == 1
    ph = o.photons()
    st = o.particles()
    assert ph["cell"][0] == st["cell"][0] and ph["off"][0] == st["off"][0]


# --- cascade growth and spectrum (Sections 3-4) ----------------------------------

def _frozen_cascade(E0, gthr, eps, lpp, dt, steps, nx=16, ppc=1, spread=0.0, lib=None):
    p = dict(nx=nx, ppc=ppc, dx=0.01, dt=dt, n0=1e-12, u_spread=spread, seed=3, E0=E0,
             gamma_thr=gthr, eps_gamma=eps, l_pp=lpp, particle_cap=2000000)
    if spread == 0.0:
        o = oracle.Oracle.from_state(p, [0, 0], [0.5, 0.5], [0.0, 0.0], [-1, 1], lib_path=lib)
    else:
        o = oracle.Oracle(p, lib)
    d = o.step(steps)
    return o, d


@pytest.mark.parametrize("lpp", [0.0, 0.1])
def test_frozen_field_growth_rate(lpp, lib=None):
    """Cascade growth in a uniform field (the Section 3 setting before
    screening) against the exact renewal root, the two-population model of
    Eq. 1-2 and the Lambert-W solution of Eq. 3."""
    E0, gthr, eps, dt = 100.0, 50.0, 10.0, 1e-3
    o, d = _frozen_cascade(E0, gthr, eps, lpp, dt, 3000 if lpp == 0 else 3500, lib=lib)
    n = d["n_elec"] + d["n_posi"]
    t = d["t"]
    G = F.growth_rate(t, n, 0.5 * t[-1], t[-1])
    delay = o.n_pp * dt
    assert G == pytest.approx(F.frozen_field_cascade_rate(E0, gthr, eps, delay), rel=0.01)
    assert G == pytest.approx(F.two_population_rate(E0, gthr, eps, delay), rel=0.10)
    if lpp == 0.0:
        assert G == pytest.approx(F.lambert_rate(E0, gthr, eps), rel=0.10)


def test_frozen_field_spectrum_slope(lib=None):
    """Eq. 7: between the pair energy and the recoil energy, the distribution
    along the accelerating direction falls as exp(-G u / E0); Eq. 8 writes the
    slope as ln(2/f)/gamma_thr."""
    E0, gthr, eps = 100.0, 50.0, 10.0
    o, d = _frozen_cascade(E0, gthr, eps, 0.0, 1e-3, 2200, nx=16, ppc=2, spread=20.0, lib=lib)
    st = o.particles()
    wv = st["q"] * st["u"]
    G = F.growth_rate(d["t"], d["n_elec"] + d["n_posi"], 1.1, 2.2)
    up = np.sqrt((eps / 2) ** 2 - 1)
    ur = np.sqrt((gthr - eps) ** 2 - 1)
    h, b = np.histogram(wv, bins=30, range=(up, ur))
    c = 0.5 * (b[1:] + b[:-1])
    slope = np.polyfit(c[1:-1], np.log(h[1:-1]), 1)[0]
    assert slope == pytest.approx(-G / E0, rel=0.10)
    assert slope == pytest.approx(-np.log(2.0 / (eps / gthr)) / gthr, rel=0.25)


# --- screening and oscillation (Sections 3 and 5) -----------------------------------

def test_screening_and_large_amplitude_oscillation(lib=None):
    """Self-consistent cascade: the field is screened with all of its energy in
    the pairs (Eq. 10 balance), the pair density lands within the factor the
    paper reports below Eq. 5 (per-species reading: a further factor 2), and
    the following uniform oscillation has the period that the measured
    momentum distribution fixes (the large-amplitude form of Eq. 11-12)."""
    E0, gthr, eps = 200.0, 100.0, 10.0
    p = dict(nx=16, ppc=4, dx=0.02, dt=0.001, n0=1.0, u_spread=0.0, seed=7, E0=E0,
             gamma_thr=gthr, eps_gamma=eps, l_pp=0.0, particle_cap=1000000)
    o = oracle.Oracle(p, lib)
    d = o.step(2500)
    t = d["t"]
    z = F.zero_crossings(t, d["E_mean"])
    ks = int(np.searchsorted(t, z[0]))
    L = p["nx"] * p["dx"]
    conv = (d["U_K"][ks] + d["U_gamma"][ks] - d["U_K"][0]) / (0.5 * E0 ** 2 * L)
    assert conv == pytest.approx(1.0, abs=5e-3)
    ns = d["n_elec"][ks] / (p["nx"] * p["ppc"])
    ratio = F.screening_density(E0, gthr, eps) / ns
    assert 1.2 < ratio < 3.0
    G = F.frozen_field_cascade_rate(E0, gthr, eps, 0.0)
    assert 0.8 < z[0] / (F.screening_time(E0, G) + 0.5 * gthr / E0) < 1.25
    # pair creation has stopped by t = 2.5: exact uniform-mode period
    assert d["n_elec"][-1] == d["n_elec"][-500]
    st = o.particles()
    w = p["n0"] * p["dx"] / p["ppc"]
    Tq = F.uniform_mode_period(d["E_mean"][-1], st["u"], st["q"], w / L)
    d2 = o.step(6000)
    Tm = 2 * np.mean(np.diff(F.zero_crossings(d2["t"], d2["E_mean"])))
    assert Tm == pytest.approx(Tq, rel=1e-3)


# --- host-side validation -------------------------------------------------------------

@pytest.mark.parametrize("bad", [
    dict(eps_gamma=1.5),                     # below the pair rest mass
    dict(gamma_thr=10.5, eps_gamma=10.0),    # recoil below gamma = 1
    dict(gamma_thr=12.0, eps_gamma=9.0),     # f >= 2/3: Eq. 1 delay not positive
    dict(dt=0.2, dx=0.1),                    # c dt >= dx
    dict(nx=1),
    dict(l_pp=-1.0),
])
def test_invalid_parameters_rejected(bad):
    p = dict(nx=16, ppc=2, dx=0.1, dt=0.05, n0=1.0, u_spread=0.0, seed=1, E0=1.0,
             gamma_thr=20.0, eps_gamma=10.0, l_pp=0.0)
    p.update(bad)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(p)


def test_capacity_error():
    p = dict(nx=16, ppc=2, dx=0.1, dt=0.05, n0=1.0, u_spread=0.0, seed=1, E0=10.0,
             gamma_thr=20.0, eps_gamma=10.0, l_pp=0.0, particle_cap=40)
    o = oracle.Oracle(p)
    with pytest.raises(oracle.OracleError, match="capacity"):
        o.step(400)
