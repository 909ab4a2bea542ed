"""Ensemble diagnostics of a cascade from its per-step records (host side).

These summarise a run the way Sections 3-6 of arXiv:2012.05587 describe it:
cascade growth rate of the pair number (Fig. 1 / Eq. 3), the peak field after
screening, the frequency of the large-amplitude oscillation of the mean field
(Section 5, Eq. 12), the damping of its envelope by secondary pair bursts
(Section 6, Eq. 24) and the final pair count.  They post-process records only.
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
    hi_frac of its final value (least squares on ln n)."""
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


def crossing_time(t, y, level) -> float:
    """First time y(t) reaches level, interpolated linearly between samples."""
    t = np.asarray(t, float)
    y = np.asarray(y, float)
    idx = np.flatnonzero(y >= level)
    if len(idx) == 0:
        return float("nan")
    i = int(idx[0])
    if i == 0:
        return float(t[0])
    return float(t[i - 1] + (level - y[i - 1]) * (t[i] - t[i - 1]) / (y[i] - y[i - 1]))


def growth_window(params: dict):
    """Particle counts between which the cascade growth rate is measured,
    fixed by the parameters alone, so every precision and seed is measured
    over the same counts: from 4 N0 (past the first generations) to N0 M / 4,
    with N0 the seed count and M = E0^2 ln(2/f) / (2 gamma_thr) the density
    at screening of Eq. 5 in units of n0 (the flattening near screening, which
    Section 3 notes, stays outside).  None when the window is narrower than a
    factor 4: the cascade is too short to have a growth phase."""
    n0 = 2.0 * params["nx"] * params["ppc"]
    M = screening_density(params["E0"], params["gamma_thr"], params["eps_gamma"]) / params.get("n0", 1.0)
    lo, hi = 4.0 * n0, n0 * M / 4.0
    return (lo, hi) if hi >= 4.0 * lo else None


def growth_rate_between(t, n, n_lo, n_hi) -> float:
    """Growth rate of n(t) from count n_lo to count n_hi: ln(n_hi / n_lo)
    over the time between the two crossings of ln n(t)."""
    lnn = np.log(np.maximum(np.asarray(n, float), 1e-300))
    t_lo = crossing_time(t, lnn, np.log(n_lo))
    t_hi = crossing_time(t, lnn, np.log(n_hi))
    if not (t_hi > t_lo):
        return float("nan")
    return float(np.log(n_hi / n_lo) / (t_hi - t_lo))


def seed_averaged_growth_rate(records: list, window) -> float:
    """Growth rate of the seed average of ln N(t) (N = electrons +
    positrons) between the counts of ``window`` (see growth_window); the
    records share their time base."""
    if window is None or not records:
        return float("nan")
    k = min(len(r["t"]) for r in records)
    lnN = np.mean([np.log((r["n_elec"] + r["n_posi"])[:k].astype(float)) for r in records], axis=0)
    return growth_rate_between(records[0]["t"][:k], np.exp(lnN), *window)


def field_peaks(t, E):
    """Times and values of the peaks of |<E>| between consecutive zeros of
    <E> (one per half period of the oscillation that follows screening)."""
    t = np.asarray(t, float)
    E = np.asarray(E, float)
    z = zero_crossings(t, E)
    tp, vp = [], []
    for a, b in zip(z[:-1], z[1:]):
        m = (t >= a) & (t <= b)
        if not m.any():
            continue
        i = int(np.argmax(np.abs(E[m])))
        tp.append(t[m][i])
        vp.append(abs(E[m][i]))
    return np.array(tp), np.array(vp)


def damping_rate(t, E, hi=0.9, lo=0.4):
    """Decay rate of the envelope of <E> after screening (Section 6, Eq. 24:
    the envelope falls as exp(-eps0 omega0 t / (4 pi)), so the rate is
    eps0 omega0 / (4 pi)).  Least-squares slope of ln |peak| against the
    peak times, over the peaks from the first one below hi P to the last one
    above lo P, P being the first peak after screening: a window fixed in
    amplitude, so the onset time of the instability does not enter.  Returns
    (rate, peaks used); a run whose envelope never falls below hi P returns
    the slope over all its peaks (an undamped run: about zero)."""
    tp, vp = field_peaks(t, E)
    if len(vp) < 3:
        return float("nan"), 0
    P = vp[0]
    below = np.flatnonzero(vp < hi * P)
    if len(below) == 0:
        return float(-np.polyfit(tp, np.log(vp), 1)[0]), len(vp)
    first = int(below[0])
    last = first
    while last + 1 < len(vp) and vp[last + 1] >= lo * P:
        last += 1
    if last - first + 1 < 3:
        return float("nan"), last - first + 1
    sl = slice(first, last + 1)
    return float(-np.polyfit(tp[sl], np.log(vp[sl]), 1)[0]), last - first + 1


def ensemble(rec: dict, params: dict | None = None) -> dict:
    """Ensemble diagnostics of one run: growth rate between the counts of
    growth_window (with params; else between 5% and 50% of the final count),
    screening time (first zero of <E>), peak |<E>| after screening,
    oscillation frequency of <E> on the plateau after screening (the first
    eight half periods: Eq. 12's omega0), damping rate of the envelope and
    Eq. 24's eps0 = 4 pi rate / omega0, final pair count and final energy."""
    t = rec["t"]
    E = rec["E_mean"]
    n = rec["n_elec"] + rec["n_posi"]
    z = zero_crossings(t, E)
    win = growth_window(params) if params is not None else None
    if params is not None:
        G = growth_rate_between(t, n, *win) if win else float("nan")
    else:
        G = growth_rate(t, n)
    zz = z[:9]
    omega = float(np.pi / np.mean(np.diff(zz))) if len(zz) > 2 else float("nan")
    lam, _ = damping_rate(t, E)
    tp, vp = field_peaks(t, E)
    out = {
        "growth_rate": G,
        "screening_time": float(z[0]) if len(z) else float("nan"),
        "peak_field_after_screening": float(np.abs(E[t >= z[0]]).max()) if len(z) else float("nan"),
        "oscillation_frequency": omega,
        "damping_rate": lam,
        "damping_eps0": float(4.0 * np.pi * lam / omega) if np.isfinite(lam) and omega > 0 else float("nan"),
        # the envelope fell through the whole fit window (to 0.4 of its first
        # peak): the damping rate is resolved, not a slope of noise
        "damping_resolved": float(len(vp) > 2 and bool((vp < 0.4 * vp[0]).any())),
        "final_pairs": float(rec["n_pairs_total"][-1]) if len(t) else float("nan"),
        "final_energy": float((rec["U_E"] + rec["U_K"] + rec["U_gamma"])[-1]) if len(t) else float("nan"),
    }
    return out


def paired_comparison(runs: list, refs: list, keys=None) -> dict:
    """Seed-by-seed comparison of two ensembles run from the same seeds
    (ensemble dicts in the same seed order): per diagnostic the two means,
    the relative difference of the means, and the standard error of that
    relative difference from the spread of the per-seed differences (a
    chaotic run departs from its twin after the parity horizon, so the means
    differ by sampling noise as well as by any bias)."""
    keys = keys or [k for k in refs[0] if k != "seed"]
    out = {}
    for k in keys:
        a = np.array([r[k] for r in runs], float)
        b = np.array([r[k] for r in refs], float)
        m = np.isfinite(a) & np.isfinite(b)
        if m.sum() < 2 or not np.isfinite(b[m].mean()) or b[m].mean() == 0:
            out[k] = {"mean": float(np.nanmean(a)), "ref_mean": float(np.nanmean(b)), "rel_err": float("nan"),
                      "rel_se": float("nan"), "n": int(m.sum())}
            continue
        d = a[m] - b[m]
        ref = b[m].mean()
        out[k] = {"mean": float(a[m].mean()), "ref_mean": float(ref), "rel_err": float(d.mean() / abs(ref)),
                  "rel_se": float(d.std(ddof=1) / np.sqrt(m.sum()) / abs(ref)), "n": int(m.sum())}
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
