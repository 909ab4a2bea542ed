"""Phase-space spectrum of the cascade on the GPU (Section 4, Eq. 7-8), read
through the on-device histogram of the C ABI.

In a uniform, unscreened field the distribution along the accelerating
direction falls as exp(-Gamma u / E0) between the pair energy and the
recoil energy (Eq. 7), and Eq. 8 writes that slope as ln(2/f) / gamma_thr.
The same pins hold for the oracle (tests/test_oracle_pins.py)."""
import numpy as np
import pytest

import fitting as F
from paper_2012_05587_gb300 import Cascade

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_frozen_field_spectrum_slope_from_device_histogram(precision):
    E0, gthr, eps = 100.0, 50.0, 10.0
    # n0 -> 1e-12: the plasma does not screen, E stays E0 (the Section 3
    # setting before screening)
    p = dict(nx=16, ppc=2, dx=0.01, dt=1e-3, n0=1e-12, u_spread=20.0, seed=3, E0=E0, gamma_thr=gthr,
             eps_gamma=eps, l_pp=0.0, particle_cap=2_000_000, precision=precision)
    steps = 2200
    up = np.sqrt((eps / 2) ** 2 - 1)   # pair members are born here
    ur = np.sqrt((gthr - eps) ** 2 - 1)  # a lepton lands here after emitting
    with Cascade(p) as c:
        c.step(steps)
        d = c.diag(steps)
        # accelerating direction: +u for positrons, -u for electrons
        h_pos = c.histogram(1, "u", 30, up, ur)
        h_ele = c.histogram(0, "u", 30, -ur, -up)[::-1]
    n = d["n_elec"] + d["n_posi"]
    assert n[-1] > 100 * n[0]
    G = F.growth_rate(d["t"], n, 1.1, 2.2)
    h = (h_pos + h_ele).astype(float)
    b = np.linspace(up, ur, 31)
    c_mid = 0.5 * (b[1:] + b[:-1])
    slope = np.polyfit(c_mid[1:-1], np.log(h[1:-1]), 1)[0]
    assert slope == pytest.approx(-G / E0, rel=0.10)
    assert slope == pytest.approx(-np.log(2.0 / (eps / gthr)) / gthr, rel=0.25)
