"""Leptons far above gamma = 1e6 (the regime of the threshold Section 8
estimates, gamma_thr ~ 7.3e7) against the FP64 oracle.

At u = 7.3e7 the spacing of FP32 is 8, so a one-word FP32 momentum drops any
push below 4 per step.  The library then keeps FP32 momenta as a compensated
pair of words (cascade_momentum_words), and tests the threshold and applies
the recoil in FP64 on the pair's sum.  These tests put a lepton just below
the threshold in a frozen uniform field (n0 -> 0) and compare the emission
step, the photon count k, the recoiled momentum and the pair that the photon
becomes with the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import Cascade, CascadeError, capi

pytestmark = pytest.mark.gpu


def _frozen(E0, dt, gamma_thr, eps_gamma, precision, **kw):
    p = dict(nx=64, ppc=1, dx=0.1, dt=dt, n0=1e-14, u_spread=0.0, seed=1, E0=E0, gamma_thr=gamma_thr,
             eps_gamma=eps_gamma, l_pp=0.0, particle_cap=64, precision=precision)
    p.update(kw)
    return p


def _oracle_params(p):
    return {k: v for k, v in p.items() if k not in ("precision", "u_words")}


def _run_both(p, u0, steps, q=1):
    sp = 1 if q > 0 else 0
    empty = {"cell": [], "off": [], "u": []}
    one = {"cell": [20], "off": [0.25], "u": [u0]}
    state = {"elec": one if sp == 0 else empty, "posi": one if sp == 1 else empty}
    ref = oracle.Oracle.from_state(_oracle_params(p), [20], [0.25], [u0], [q])
    d_ref = ref.step(steps)
    pr = ref.particles()
    with Cascade(p, state=state) as c:
        c.step(steps)
        d = c.diag(steps)
        parts = (c.particles(0), c.particles(1))
    return d, d_ref, parts, pr


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fine"])
def test_emission_at_the_threshold_of_section_8(precision):
    """gamma_thr = 72,999,996, f = 0.01: a positron from u0 = 72,999,840
    gains exactly 8 per step (E0 = 1024, dt = 1/128), so it reaches
    u = 7.3e7 >= gamma_thr on step 20 in any precision, emits one photon of
    eps = 729,999.96 and recoils; the photon becomes a pair in place at the
    start of step 21.  Every quantity is compared with the oracle's."""
    p = _frozen(1024.0, 1.0 / 128.0, 72_999_996.0, 729_999.96, precision)
    if precision != "fp64":
        assert capi.cascade_momentum_words(p) == 2
        with pytest.raises(CascadeError) as ei:
            capi.cascade_momentum_words(dict(p, u_words=1))
        assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG and "2^-12" in str(ei.value)
    d, d_ref, (e, q), pr = _run_both(p, 72_999_840.0, 25)
    for f in ("n_elec", "n_posi", "n_photon", "n_pairs_total", "n_emit_multi"):
        assert np.array_equal(d[f], d_ref[f]), f
    assert int(np.argmax(d_ref["n_pairs_total"] > 0)) == 20  # record of step 21
    assert d_ref["n_pairs_total"][-1] == 1
    # the recoiled positron, then the pair's electron and positron (FP32: the
    # field is gathered in FP32, so each push carries a relative rounding of
    # about 1e-7 of itself; gamma, and with it U_K, is an FP32 value)
    rtol = 1e-12 if precision == "fp64" else 1e-9
    np.testing.assert_allclose(q["u"][0], pr["u"][0], rtol=rtol)
    np.testing.assert_allclose(e["u"][0], pr["u"][1], rtol=rtol)
    np.testing.assert_allclose(q["u"][1], pr["u"][2], rtol=rtol)
    assert q["cell"][0] == pr["cell"][0] and e["cell"][0] == pr["cell"][1]
    np.testing.assert_allclose(d["U_K"], d_ref["U_K"], rtol=1e-12 if precision == "fp64" else 1e-6)
    np.testing.assert_allclose(d["U_gamma"], d_ref["U_gamma"], rtol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_electron_at_gamma_2e6_with_a_push_below_the_fp32_spacing(precision):
    """gamma_thr = 2e6 and a push of 0.1 per step against an FP32 spacing of
    0.125 at u = 2e6: one FP32 word would not move at all.  An electron from
    u0 = -(2e6 - 5.05) crosses the threshold on step 51 (the margin, 0.05,
    is far above the rounding of the pushes), emits k = 1, keeps its
    direction, and its pair is born moving along -x."""
    p = _frozen(10.0, 0.01, 2.0e6, 2.0e4, precision)
    if precision == "fp32":
        assert capi.cascade_momentum_words(p) == 2
    u0 = -(2.0e6 - 5.05)
    d, d_ref, (e, q), pr = _run_both(p, u0, 60, q=-1)
    for f in ("n_elec", "n_posi", "n_photon", "n_pairs_total"):
        assert np.array_equal(d[f], d_ref[f]), f
    assert int(np.argmax(d_ref["n_photon"] > 0)) == 50  # record of step 51
    rtol = 1e-12 if precision == "fp64" else 1e-9
    np.testing.assert_allclose(e["u"], pr["u"][pr["q"] < 0], rtol=rtol)
    np.testing.assert_allclose(q["u"], pr["u"][pr["q"] > 0], rtol=rtol)
    assert e["u"][0] < 0 and q["u"][0] < 0


def test_two_word_momenta_track_the_oracle_more_closely():
    """The small cascade with one-word and with two-word FP32 momenta
    (u_words = 2 forced): after 100 steps, through the first emissions and
    conversions, the momenta of the seed particles are closer to the FP64
    oracle's with two words (the push then loses only the FP32 rounding of
    q dt E, not half the spacing of u)."""
    from paper_2012_05587_gb300 import workloads as W

    p = W.small_cascade(precision="fp32")
    steps = 100
    ref = oracle.Oracle({k: v for k, v in p.items() if k not in ("precision", "steps")})
    ref.step(steps)
    pr = ref.particles()
    nseed = p["nx"] * p["ppc"]
    errs = {}
    for words in (1, 2):
        with Cascade(dict(p, u_words=words)) as c:
            c.step(steps)
            errs[words] = max(np.abs(c.particles(s)["u"][:nseed] - pr["u"][s:2 * nseed:2]).max() for s in (0, 1))
    assert errs[2] < 0.25 * errs[1], errs
    assert errs[2] < 1e-5, errs
