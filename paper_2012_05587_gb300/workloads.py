"""Seeded synthetic workloads: the cascade configurations, as parameter sets.

Every input of the method is an initial-value problem fixed by these numbers
(the seed keys the counter-based generator that draws the seed momenta on
each side).  Nothing here computes any step of the method.  Seeds follow
1234 + 1000 * config + run.
"""
from __future__ import annotations

import math

import numpy as np


def seed_of(config: int, run: int = 0) -> int:
    return 1234 + 1000 * config + run


def small_cascade(run: int = 0, precision: str = "fp64") -> dict:
    """Plain small cascade: Nx = 256, dx = 0.1, dt = 0.05, 16 + 16 per cell,
    u ~ N(0, 0.01), E0 = 10, gamma_thr = 20, eps_gamma = 10, l_pp = 1.0, 1000 steps."""
    return dict(nx=256, ppc=16, dx=0.1, dt=0.05, n0=1.0, u_spread=0.01, seed=seed_of(1, run), E0=10.0,
                gamma_thr=20.0, eps_gamma=10.0, l_pp=1.0, particle_cap=1 << 17, precision=precision,
                steps=1000)


def large_cascade(run: int = 0, precision: str = "fp32") -> dict:
    """Large single cascade: Nx = 16384, dx = 0.05, dt = 0.025, 64 + 64 per cell,
    E0 = 100, gamma_thr = 50, eps_gamma = 20, l_pp = 0.5, 20000 steps,
    particle cap 5e8 in total (2.5e8 per species)."""
    return dict(nx=16384, ppc=64, dx=0.05, dt=0.025, n0=1.0, u_spread=0.01, seed=seed_of(2, run), E0=100.0,
                gamma_thr=50.0, eps_gamma=20.0, l_pp=0.5, particle_cap=250_000_000, precision=precision,
                steps=20000)


def damping_cascade(run: int = 0, precision: str = "fp32", nx: int = 2048) -> dict:
    """The f = 0.1 cascade whose oscillation Sections 5-6 follow through its
    damping: Nx = 2048 (L = 41 c/omega_p), dx = 0.02, dt = 0.005, 4 + 4 seed
    particles per cell, u ~ N(0, 0.01), E0 = 100, gamma_thr = 50,
    eps_gamma = 5 (f = 0.1), in-place pairs (l_pp = 0), 10000 steps (t = 50):
    the cascade screens the field at t = 1.6, the oscillation keeps its
    amplitude for several periods, then the instability of Section 5 drives
    secondary bursts once per period and the envelope decays (Eq. 24)."""
    return dict(nx=nx, ppc=4, dx=0.02, dt=0.005, n0=1.0, u_spread=0.01, seed=seed_of(7, run), E0=100.0,
                gamma_thr=50.0, eps_gamma=5.0, l_pp=0.0, particle_cap=nx * 4 * 400, precision=precision,
                steps=10000, diag_ring=10000)


def paper_scale(f: float, precision: str = "fp32", dt_factor: float = 1.0) -> dict:
    """Section 3 setup at the paper's own parameters: E0 = 10^3.5, L = 10^1.5
    in N_L = 2000 cells, dt = 10^-3.5 (times dt_factor, for convergence
    studies), gamma_thr = 500, eps_gamma = f gamma_thr, one particle per cell
    per species at rest, in-place pair creation (l_pp = 0).  The particle
    cap allows 1.5 times the density at screening of Eq. 5."""
    g = 500.0
    E0 = 10 ** 3.5
    nx = 2000
    pred = E0 * E0 * math.log(2 / f) / (2 * g)  # Eq. 5, per species, in n0
    return dict(nx=nx, ppc=1, dx=10 ** 1.5 / nx, dt=10 ** -3.5 * dt_factor, n0=1.0, u_spread=0.0,
                seed=9000 + int(1e4 * f), E0=E0, gamma_thr=g, eps_gamma=f * g, l_pp=0.0, precision=precision,
                particle_cap=int(1.5 * pred * nx) + 4096, diag_ring=1 << 16)


def sweep_dt(E0: float, eps_gamma: float) -> float:
    """Time step of the precision sweep and the batch: resolve t_p = eps/E0 by 10."""
    return min(0.05, 0.1 * eps_gamma / E0)


def precision_sweep(run: int = 0, precision: str = "fp32") -> list:
    """Nx = 4096, 32 per species per cell, E0 in {10, 100, 1000}, gamma_thr in
    {20, 200, 2000}, eps = gamma_thr / 2, l_pp = 1, 5000 steps, dt from sweep_dt,
    dx = 2 dt; every step's record is kept (diag_ring > steps), since the
    cascade and screening happen in the first steps."""
    out = []
    for E0 in (10.0, 100.0, 1000.0):
        for g in (20.0, 200.0, 2000.0):
            eps = g / 2
            dt = sweep_dt(E0, eps)
            out.append(dict(nx=4096, ppc=32, dx=2 * dt, dt=dt, n0=1.0, u_spread=0.01, seed=seed_of(3, run),
                            E0=E0, gamma_thr=g, eps_gamma=eps, l_pp=1.0, particle_cap=250_000_000,
                            precision=precision, steps=5000, diag_ring=8192))
    return out


def predicted_particles(p: dict) -> float:
    """Both species at the end of the cascade, from the screening density of
    Eq. 5 (ln 2 for f = 1/2): 2 Nx ppc max(1, 0.693 E0^2 / gamma_thr)."""
    return 2 * p["nx"] * p["ppc"] * max(1.0, 0.693 * p["E0"] ** 2 / p["gamma_thr"])


def batch_scan(n: int = 256, run: int = 0, precision: str = "fp32", steps: int = 3000,
               max_particles: int = 1 << 25) -> list:
    """Parameter scan: Nx log-uniform in [256, 8192], ppc in {8, 16, 32, 64},
    E0 and gamma_thr log-uniform in [10, 1000], eps = gamma_thr / 2 (>= 2),
    l_pp uniform in [0.2, 2], dt from sweep_dt, dx = 2 dt.  Draws whose
    predicted particle count exceeds max_particles are redrawn from the same
    seeded stream."""
    rng = np.random.default_rng(seed_of(4, run))
    out = []
    while len(out) < n:
        nx = int(round(math.exp(rng.uniform(math.log(256), math.log(8192)))))
        ppc = int(rng.choice([8, 16, 32, 64]))
        E0 = float(math.exp(rng.uniform(math.log(10), math.log(1000))))
        g = float(math.exp(rng.uniform(math.log(10), math.log(1000))))
        lpp = float(rng.uniform(0.2, 2.0))
        eps = max(2.0, g / 2)
        if g - eps < 1.0 or eps / g >= 2.0 / 3.0:
            continue
        dt = sweep_dt(E0, eps)
        p = dict(nx=nx, ppc=ppc, dx=2 * dt, dt=dt, n0=1.0, u_spread=0.01, seed=seed_of(4, run) + len(out),
                 E0=E0, gamma_thr=g, eps_gamma=eps, l_pp=lpp, precision=precision, steps=steps)
        pred = predicted_particles(p)
        if pred > max_particles:
            continue
        p["particle_cap"] = int(min(max_particles, 1.5 * pred / 2 + nx * ppc)) + 64
        out.append(p)
    return out


def serving_requests(n: int = 2000, rate: float = 50.0, run: int = 0, precision: str = "fp32") -> list:
    """Poisson arrivals (mean rate req/s) of requests drawn from the batch-scan
    distribution with steps uniform in [500, 5000]."""
    rng = np.random.default_rng(seed_of(5, run))
    base = batch_scan(n, run=run, precision=precision)
    t = 0.0
    out = []
    for p in base:
        t += float(rng.exponential(1.0 / rate))
        q = dict(p)
        q["steps"] = int(rng.integers(500, 5001))
        q["arrival"] = t
        out.append(q)
    return out


def corotating(nx: int = 10000, precision: str = "fp32", gamma_thr: float = 5000.0, eps_gamma: float = 50.0,
               dt: float = 1e-3, dx: float = 0.1, ppc: int = 4, l_pp: float = 0.0) -> dict:
    """Co-rotating-frame run of Section 7, in units of n_GJ = |rho_GJ| / e and
    omega_p,GJ: L = nx dx (1000 in the paper), dx = 0.1, dt = 1e-3, open
    boundaries, rho_GJ = -1, j_m = -1.5 rho_GJ c = 1.5, gamma_thr = 5000,
    f = 0.01.  ppc is the positron count per cell (electrons: 2 ppc), so the
    weight n0 dx / ppc with n0 = 1 gives densities 2 and 1."""
    return dict(nx=nx, ppc=ppc, dx=dx, dt=dt, n0=1.0, u_spread=0.0, seed=seed_of(6), E0=0.0,
                gamma_thr=gamma_thr, eps_gamma=eps_gamma, l_pp=l_pp, j_m=1.5, rho_gj=-1.0, open_bc=1,
                precision=precision, particle_cap=max(1 << 20, 64 * nx * ppc), diag_ring=1 << 16)


def corotating_state(p: dict):
    """Cold initial state of Section 7: electrons of density 2 and positrons
    of density 1, evenly spaced (rho = rho_GJ = -1, so E = 0 satisfies
    Gauss's law), drifting with v = -1/2 and +1/2 so that the current equals
    j_m = 1.5.  Returns ((cell, offset, u, q) arrays, E)."""
    nx, ppc = p["nx"], p["ppc"]
    v = 0.5
    u = v / math.sqrt(1.0 - v * v)
    cells, offs, us, qs = [], [], [], []
    for n, uu, q in ((2 * ppc, -u, -1), (ppc, u, 1)):
        i = np.repeat(np.arange(nx), n)
        k = np.tile(np.arange(n), nx)
        cells.append(i)
        offs.append((k + 0.5) / n)
        us.append(np.full(len(i), uu))
        qs.append(np.full(len(i), q))
    state = (np.concatenate(cells).astype(np.int32), np.concatenate(offs), np.concatenate(us),
             np.concatenate(qs).astype(np.int8))
    return state, np.zeros(nx)
