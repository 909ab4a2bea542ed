"""Pins of the oracle's co-rotating-frame terms and open boundaries
(Section 7, Eq. 25-26): the background current j_m in Ampere's law, the
background charge rho_GJ in Gauss's law, and particles leaving the domain."""
import numpy as np
import pytest

import fitting as F
import oracle


def cold_state(nx, per_cell_e, per_cell_p, u_e, u_p):
    """Evenly spaced electrons and positrons (per_cell_* per cell), cold."""
    cells, offs, us, qs = [], [], [], []
    for n, u, q in ((per_cell_e, u_e, -1), (per_cell_p, u_p, 1)):
        i = np.repeat(np.arange(nx), n)
        k = np.tile(np.arange(n), nx)
        cells.append(i)
        offs.append((k + 0.5) / n)
        us.append(np.full(len(i), u))
        qs.append(np.full(len(i), q))
    return np.concatenate(cells), np.concatenate(offs), np.concatenate(us), np.concatenate(qs)


def base(**kw):
    p = dict(nx=16, ppc=2, dx=0.1, dt=0.01, n0=1.0, u_spread=0.0, seed=1, E0=0.0, gamma_thr=1e9,
             eps_gamma=10.0, l_pp=0.0, j_m=0.0, rho_gj=0.0, open_bc=0)
    p.update(kw)
    return p


def test_background_current_drives_the_uniform_mode(lib=None):
    """A cold plasma at rest with electron density 2 and positron density 1
    (w = n0 dx / ppc with ppc = the positron count): dE/dt = -(J - j_m) gives
    E^1 = dt j_m and E^{n+1} - 2 E^n + E^{n-1} = -w_p^2 dt^2 E^n with
    w_p^2 = 2 + 1, so E^n = A sin(n theta), 2 - 2 cos(theta) = 3 dt^2,
    A sin(theta) = dt j_m."""
    dt, jm = 0.01, 1e-5
    p = base(dt=dt, j_m=jm)
    c, o, u, q = cold_state(16, 4, 2, 0.0, 0.0)
    orc = oracle.Oracle.from_state(p, c, o, u, q, E=np.zeros(16), lib_path=lib)
    d = orc.step(8000)
    theta = np.arccos(1.0 - 1.5 * dt * dt)
    A = dt * jm / np.sin(theta)
    n = d["step"]
    want = A * np.sin(n * theta)
    assert np.abs(d["E_mean"] - want).max() <= 1e-6 * A
    w = 2 * np.pi / F.period_from_crossings(d["t"], d["E_mean"])
    assert w == pytest.approx(theta / dt, rel=1e-7)


def test_corotating_equilibrium_is_stationary(lib=None):
    """Section 7 initial state on a periodic grid: rho_- = -2, rho_+ = +1,
    so rho = rho_GJ = -1 and E = 0 satisfies Eq. 25; drifts v_- = -1/2,
    v_+ = +1/2 give J = 2/2 + 1/2 = 3/2 = j_m = -1.5 rho_GJ, so Eq. 26 keeps
    E = 0."""
    v = 0.5
    uu = v / np.sqrt(1 - v * v)
    p = base(dt=0.01, j_m=1.5, rho_gj=-1.0, ppc=4)  # w = n0 dx / 4: 8 e- and 4 e+ per cell
    c, o, u, q = cold_state(16, 8, 4, -uu, uu)
    orc = oracle.Oracle.from_state(p, c, o, u, q, E=np.zeros(16), lib_path=lib)
    d = orc.step(2000)
    assert np.abs(d["E_absmax"]).max() <= 1e-10
    assert np.abs(d["gauss_resid"]).max() <= 1e-12
    assert np.all(d["n_elec"] == 128) and np.all(d["n_posi"] == 64)


def test_open_boundary_removes_departing_particles(lib=None):
    """A positron crossing x = L and an electron crossing x = 0 leave in the
    step they cross (frozen field).  The initial E = 0 does not satisfy
    Gauss's law for their charges; the interior residual stays at its
    initial value (charge conservation through the boundary)."""
    dt, dx = 0.01, 0.1
    p = base(nx=20, dx=dx, dt=dt, n0=1e-12, open_bc=1)
    u = 3.0
    v = u / np.sqrt(1 + u * u)
    steps_to_cross = int(np.floor(0.5 * dx / (v * dt))) + 1  # from offset 0.5 of the edge cell
    orc = oracle.Oracle.from_state(p, [19, 0], [0.5, 0.5], [u, -u], [1, -1], lib_path=lib)
    r0 = orc.diag_now()["gauss_resid"]
    assert r0 > 0
    d = orc.step(steps_to_cross - 1)
    assert d["n_posi"][-1] == 1 and d["n_elec"][-1] == 1
    d = orc.step(1)
    assert d["n_posi"][-1] == 0 and d["n_elec"][-1] == 0
    assert d["gauss_resid"][-1] == pytest.approx(r0, rel=1e-12)


def test_open_boundary_outflow_keeps_gauss(lib=None):
    """A drifting positron beam streams out through x = L with its
    self-consistent field, starting from the E that satisfies Gauss's law
    (E_{i+1/2} = (i + 1/2) dx for density 1, so node i sits between edges
    whose difference is dx); the interior residual stays at round-off while
    charge leaves."""
    nx, dx = 64, 0.1
    p = base(nx=nx, dx=dx, dt=0.02, open_bc=1, n0=1.0, ppc=4)
    c, o, u, q = cold_state(nx, 0, 4, 0.0, 0.8)
    E = (np.arange(nx) + 0.5) * dx
    orc = oracle.Oracle.from_state(p, c, o, u, q, E=E, lib_path=lib)
    assert orc.diag_now()["gauss_resid"] <= 1e-14
    d = orc.step(600)
    assert d["n_posi"][-1] < d["n_posi"][0] / 2
    assert np.abs(d["gauss_resid"]).max() <= 1e-12 * np.abs(d["E_absmax"]).max()


def test_open_boundary_gather_uses_the_edge_field(lib=None):
    """At rest in cell 0 below the middle, the particle sits between x = 0 and
    the first edge: with open boundaries both gather points read E[0]."""
    p = base(nx=8, dx=0.1, dt=0.01, n0=1e-12, open_bc=1)
    E = np.linspace(1.0, 8.0, 8)
    orc = oracle.Oracle.from_state(p, [0], [0.2], [0.0], [1], E=E, lib_path=lib)
    orc.step(1)
    assert orc.particles()["u"][0] == pytest.approx(0.01 * E[0], rel=1e-14)
    periodic = oracle.Oracle.from_state(dict(p, open_bc=0), [0], [0.2], [0.0], [1], E=E, lib_path=lib)
    periodic.step(1)
    assert periodic.particles()["u"][0] != pytest.approx(0.01 * E[0], rel=1e-3)


def test_open_boundary_drops_photons_converting_outside(lib=None):
    """Emission near x = L with l_pp pointing out of the domain: the photon is
    not kept; the same emission pointing inward is."""
    p = base(nx=20, dx=0.1, dt=0.01, n0=1e-14, E0=1.0, gamma_thr=20.0, eps_gamma=4.0, l_pp=0.55, open_bc=1)
    out = oracle.Oracle.from_state(p, [19], [0.2], [19.99], [1], lib_path=lib)
    d = out.step(1)
    assert d["n_photon"][0] == 0 and d["n_posi"][0] == 1
    inward = oracle.Oracle.from_state(p, [19], [0.2], [-19.99], [1], E=np.full(20, -1.0), lib_path=lib)
    d = inward.step(1)
    assert d["n_photon"][0] == 1
