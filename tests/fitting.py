"""Closed forms and fits used by the tests (host-side analysis only).

Nothing here steps a cascade; these are the analytic results of
arXiv:2012.05587 and of the textbook special cases of the same equations,
written out so the oracle and the CUDA path can be checked against them.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq
from scipy.special import lambertw

from paper_2012_05587_gb300 import analysis as _analysis


# --- time-series measurements ------------------------------------------------

def zero_crossings(t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Times where y changes sign, from a cubic through the 4 samples around each."""
    out = []
    for i in range(1, len(y) - 2):
        if y[i] == 0.0:
            out.append(t[i])
            continue
        if y[i] * y[i + 1] < 0:
            ts = t[i - 1:i + 3]
            ys = y[i - 1:i + 3]
            c = np.polyfit(ts - t[i], ys, 3)
            roots = np.roots(c)
            h = t[i + 1] - t[i]
            good = [r.real + t[i] for r in roots if abs(r.imag) < 1e-12 and -1e-12 <= r.real <= h + 1e-12]
            if good:
                out.append(min(good, key=lambda r: abs(r - t[i] - h / 2)))
            else:  # fall back to linear interpolation
                out.append(t[i] - y[i] * h / (y[i + 1] - y[i]))
    return np.array(out)


def period_from_crossings(t, y) -> float:
    z = zero_crossings(np.asarray(t, float), np.asarray(y, float))
    if len(z) < 3:
        raise ValueError("need at least three zero crossings")
    return 2.0 * (z[-1] - z[0]) / (len(z) - 1)


def growth_rate(t, n, t0, t1) -> float:
    """Least-squares slope of ln n(t) over [t0, t1]."""
    t = np.asarray(t, float)
    n = np.asarray(n, float)
    m = (t >= t0) & (t <= t1) & (n > 0)
    return float(np.polyfit(t[m], np.log(n[m]), 1)[0])


# --- closed forms -------------------------------------------------------------

def leapfrog_uniform_mode_omega(n0: float, dt: float) -> float:
    """Cold, non-relativistic uniform mode of a pair plasma (n0 per species, so
    the continuum frequency is sqrt(2 n0)) under the leapfrog push + Ampere
    update: 2 sin(omega dt / 2) / dt = sqrt(2 n0)."""
    return 2.0 / dt * np.arcsin(dt * np.sqrt(2.0 * n0) / 2.0)


def relativistic_uniform_mode_period(E0: float, n0: float) -> float:
    """Period of the cold, uniform, relativistic pair-plasma oscillation started
    from u = 0 in field E0 (n0 per species).

    du/dt = E for positrons (electrons mirror them), dE/dt = -2 n0 u / gamma,
    so E^2 = E0^2 - 4 n0 (gamma - 1) and a quarter period is the integral of
    du / E(u) from 0 to u_max, gamma_max = 1 + E0^2 / (4 n0)."""
    gm = 1.0 + E0 * E0 / (4.0 * n0)
    um = np.sqrt(gm * gm - 1.0)

    def integrand(phi):
        u = um * np.sin(phi)
        g = np.sqrt(1.0 + u * u)
        e2 = E0 * E0 - 4.0 * n0 * (g - 1.0)
        return um * np.cos(phi) / np.sqrt(max(e2, 1e-300))

    val, _ = quad(integrand, 0.0, np.pi / 2, epsabs=1e-13, epsrel=1e-12, limit=400)
    return 4.0 * val


# Exact growth rate of the threshold cascade in a frozen uniform field (the
# renewal equation of the model's lepton generations; reduces to Eq. 3 for
# f << 1): one copy, shared with the benchmark's reports.
frozen_field_cascade_rate = _analysis.renewal_growth_rate


def two_population_rate(E0, gamma_thr, eps_gamma, delay=0.0) -> float:
    """Growth rate of the two-population model, Eq. 1 and Eq. 2, solved with
    exp(G t) trial solutions without the f << 1 step:
        exp(G tau) = 1 + 2 (1 - f) exp(-G d) / (f t_a (G + 1/tau)),
    tau = (1 - 3 f / 2) t_a, t_a = gamma_thr / E0, f = eps_gamma / gamma_thr;
    d is the photon flight delay (zero in the paper)."""
    f = eps_gamma / gamma_thr
    ta = gamma_thr / E0
    tau = (1.0 - 1.5 * f) * ta

    def fn(G):
        return np.exp(G * tau) - 1.0 - 2.0 * (1.0 - f) * np.exp(-G * delay) / (f * ta * (G + 1.0 / tau))

    return brentq(fn, 1e-9 / ta, 100.0 / ta)


def lambert_rate(E0, gamma_thr, eps_gamma) -> float:
    """Eq. 3: G t_a = W(2 / f)."""
    f = eps_gamma / gamma_thr
    return float(lambertw(2.0 / f).real) * E0 / gamma_thr


def screening_density(E0, gamma_thr, eps_gamma) -> float:
    """Eq. 5 in units of n0: n_s = E0^2 ln(2/f) / (2 gamma_thr)."""
    f = eps_gamma / gamma_thr
    return E0 * E0 * np.log(2.0 / f) / (2.0 * gamma_thr)


def screening_time(E0, G, n0=1.0) -> float:
    """Section 3: t_s = ln(E0 G / (2 n0)) / G (the 8 pi e c n0 of the paper is
    2 n0 in these units)."""
    return np.log(E0 * G / (2.0 * n0)) / G


def uniform_mode_period(E_start: float, u: np.ndarray, q: np.ndarray, w_over_L: float) -> float:
    """Exact period of a spatially uniform plasma oscillation for an arbitrary
    momentum distribution (no pair creation).

    With E uniform, every particle obeys du/dt = q E, so u_p(t) = u_p + q A(t)
    with dA/dt = E, and the energy E^2/2 + sum_p (w/L) gamma_p is conserved
    (Ampere dE/dt = -J with J the mean current).  Hence
        (dA/dt)^2 = V(A) = E_start^2 - 2 (w/L) sum_p [gamma(u_p + q_p A) - gamma(u_p)],
    and A swings between the two roots of V; the period is twice the integral
    of dA / sqrt(V) between them.  Eq. 11 and Eq. 12 are the small-amplitude
    limit of this (V quadratic, curvature 2 n <1/gamma^3>)."""
    u = np.asarray(u, float)
    q = np.asarray(q, float)
    g0 = np.sqrt(1.0 + u * u).sum()

    def V(A):
        return E_start * E_start - 2.0 * w_over_L * (np.sqrt(1.0 + (u + q * A) ** 2).sum() - g0)

    # bracket the turning points
    step = max(abs(E_start), 1e-6)
    hi = step
    while V(hi) > 0:
        hi *= 2.0
    lo = -step
    while V(lo) > 0:
        lo *= 2.0
    a_plus = brentq(V, 0.0, hi, xtol=1e-14, rtol=1e-15)
    a_minus = brentq(V, lo, 0.0, xtol=1e-14, rtol=1e-15)
    mid = 0.5 * (a_plus + a_minus)
    half = 0.5 * (a_plus - a_minus)

    def integrand(phi):
        A = mid + half * np.sin(phi)
        v = V(A)
        return half * np.cos(phi) / np.sqrt(v) if v > 0 else 0.0

    val, _ = quad(integrand, -np.pi / 2, np.pi / 2, epsabs=1e-12, epsrel=1e-10, limit=400)
    return 2.0 * val
