"""Ensemble diagnostics of a cascade from its per-step records (host side).

These summarise a run the way Sections 3-6 of arXiv:2012.05587 describe it:
cascade growth rate of the pair number (Fig. 1 / Eq. 3), the peak field after
screening, the frequency of the large-amplitude oscillation of the mean field
(Section 5) and the final pair count.  They post-process records only.
"""
from __future__ import annotations

import numpy as np


def zero_crossings(t, y) -> np.ndarray:
    t = np.asarray(t, float)
    y = np.asarray(y, float)
    s = np.signbit(y)
    idx = np.flatnonzero(s[1:] != s[:-1])
    # linear interpolation between the bracketing samples
    return t[idx] - y[idx] * (t[idx + 1] - t[idx]) / (y[idx + 1] - y[idx])


def growth_rate(t, n, lo_frac=0.05, hi_frac=0.5) -> float:
    """Exponential growth rate of n(t) while it rises from lo_frac to
    hi_frac of its final value (the cascade phase before screening)."""
    t = np.asarray(t, float)
    n = np.asarray(n, float)
    if len(n) < 3 or n[-1] <= n[0]:
        return float("nan")
    lo = n[0] + lo_frac * (n[-1] - n[0])
    hi = n[0] + hi_frac * (n[-1] - n[0])
    m = (n >= lo) & (n <= hi)
    if m.sum() < 3:
        return float("nan")
    return float(np.polyfit(t[m], np.log(n[m]), 1)[0])


def ensemble(rec: dict) -> dict:
    """Growth rate, screening time, peak |<E>| after screening, oscillation
    frequency of <E>, final pair count and final energy of one run."""
    t = rec["t"]
    E = rec["E_mean"]
    n = rec["n_elec"] + rec["n_posi"]
    z = zero_crossings(t, E)
    out = {
        "growth_rate": growth_rate(t, n),
        "screening_time": float(z[0]) if len(z) else float("nan"),
        "peak_field_after_screening": float(np.abs(E[t >= z[0]]).max()) if len(z) else float("nan"),
        "oscillation_frequency": float(np.pi / np.mean(np.diff(z))) if len(z) > 2 else float("nan"),
        "final_pairs": float(rec["n_pairs_total"][-1]) if len(t) else float("nan"),
        "final_energy": float((rec["U_E"] + rec["U_K"] + rec["U_gamma"])[-1]) if len(t) else float("nan"),
    }
    return out


def relative_errors(a: dict, ref: dict) -> dict:
    out = {}
    for k, v in ref.items():
        x = a.get(k, float("nan"))
        out[k] = float(abs(x - v) / abs(v)) if v not in (0.0,) and np.isfinite(v) and np.isfinite(x) else float("nan")
    return out


# --- closed forms of the model (Sections 3-5) ------------------------------------

def lambert_growth_rate(E0: float, gamma_thr: float, eps_gamma: float) -> float:
    """Eq. 3: Gamma t_a = W(2/f), t_a = gamma_thr / E0."""
    from scipy.special import lambertw

    f = eps_gamma / gamma_thr
    return float(lambertw(2.0 / f).real) * E0 / gamma_thr


def renewal_growth_rate(E0: float, gamma_thr: float, eps_gamma: float, delay: float = 0.0) -> float:
    """Exact growth rate of the threshold cascade in a frozen uniform field.

    In a uniform field u grows linearly, so a lepton at the threshold
    (u_thr = sqrt(gamma_thr^2 - 1)) that recoils to gamma_thr - eps (u_r) emits
    again after T1 = (u_thr - u_r) / E0.  Each photon becomes, after the flight
    delay d, two leptons of gamma = eps / 2 (u_p) moving along it (Section 2):
    the one whose charge the field accelerates forward reaches the threshold
    after T2 = (u_thr - u_p) / E0, the other turns around and needs
    T3 = (u_thr + u_p) / E0.  Counting descendants (Euler-Lotka) gives
        exp(-G (T2 + d)) + exp(-G (T3 + d)) = 1 - exp(-G T1).
    For f << 1 and d = 0 this reduces to Eq. 3."""
    from scipy.optimize import brentq

    ut = np.sqrt(gamma_thr ** 2 - 1.0)
    ur = np.sqrt((gamma_thr - eps_gamma) ** 2 - 1.0)
    up = np.sqrt((eps_gamma / 2.0) ** 2 - 1.0)
    T1, T2, T3 = (ut - ur) / E0, (ut - up) / E0, (ut + up) / E0
    return float(brentq(lambda G: np.exp(-G * (T2 + delay)) + np.exp(-G * (T3 + delay)) - (1 - np.exp(-G * T1)),
                        1e-9 / T1, 50.0 / T1))


def screening_density(E0: float, gamma_thr: float, eps_gamma: float) -> float:
    """Eq. 5 in units of n0."""
    return E0 * E0 * np.log(2.0 * gamma_thr / eps_gamma) / (2.0 * gamma_thr)


def mean_gamma(gamma_thr: float, eps_gamma: float) -> float:
    """Eq. 10: <gamma> = gamma_thr / ln(2/f)."""
    return gamma_thr / np.log(2.0 * gamma_thr / eps_gamma)
