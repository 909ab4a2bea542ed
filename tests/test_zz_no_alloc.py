"""The allocation-free Gauss check against the allocating one and the oracle.

cascade_gauss_noalloc serves callers that cannot allocate device memory
(applications that reserve all device memory for their own pool, plug-ins
whose host program owns every allocation, real-time loops that may not call
cudaMalloc); it keeps its scratch in a static device array instead.  Here it
reads the same state as cascade_gauss, from device buffers the test owns, and
must return the same residual, on two calls in a row (the second call finds
the first one's data in the shared scratch and must clear it).  The oracle's
residual of the same state (FP64) is the third witness.  This file is
collected last so that a stopping run has executed every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import Cascade, CascadeError, capi, workloads as W

pytestmark = pytest.mark.gpu

GAUSS_RTOL = 1e-12  # the FP64 tolerance the Gauss-law tests use
PREC = {"fp64": capi.CASCADE_FP64, "fp32": capi.CASCADE_FP32_MIXED, "fp32_fine": capi.CASCADE_FP32_MIXED_FINE}


def _oracle_params(p):
    return {k: v for k, v in p.items() if k not in ("precision", "steps", "photon_cap", "diag_ring")}


def _device_state(parts, E_host, precision):
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    dt = torch.float64 if precision == "fp64" else torch.float32
    return {
        "cell_e": torch.as_tensor(parts[0]["cell"], dtype=torch.int32, device=dev),
        "off_e": torch.as_tensor(parts[0]["off"], dtype=dt, device=dev),
        "cell_p": torch.as_tensor(parts[1]["cell"], dtype=torch.int32, device=dev),
        "off_p": torch.as_tensor(parts[1]["off"], dtype=dt, device=dev),
        "E": torch.as_tensor(E_host, dtype=torch.float64, device=dev),
    }


def _noalloc(p, parts, d, precision):
    import torch

    w = p["n0"] * p["dx"] / p["ppc"]
    torch.cuda.synchronize()
    return capi.cascade_gauss_noalloc(
        p["nx"], p["dx"], w, PREC[precision], len(parts[0]["cell"]), d["cell_e"].data_ptr(), d["off_e"].data_ptr(),
        len(parts[1]["cell"]), d["cell_p"].data_ptr(), d["off_p"].data_ptr(), d["E"].data_ptr(),
        torch.cuda.current_stream().cuda_stream, rho_gj=p.get("rho_gj", 0.0), open_bc=p.get("open_bc", 0))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fine"])
def test_noalloc_gauss_matches_allocating_entry_point(precision):
    p = dict(W.small_cascade(), precision=precision)
    rng = np.random.default_rng(42)
    with Cascade(p) as seed_run:
        seed_run.step(40)  # particles spread over the grid and gain momentum
        parts = [seed_run.particles(s) for s in (0, 1)]
        E_run, _ = seed_run.fields()
    # a field that does not satisfy Gauss's law, so the residual is O(1) and
    # both implementations must agree on its value, not just on "small"
    E_host = E_run + rng.normal(0.0, 0.5, p["nx"])
    state = {"elec": parts[0], "posi": parts[1], "E": E_host}
    with Cascade(p, state=state) as c:
        r_ref = c.gauss()
        d = _device_state(parts, E_host, precision)
        results = [_noalloc(p, parts, d, precision) for _ in range(2)]
    assert r_ref > 0.1
    for r in results:
        assert r == pytest.approx(r_ref, rel=GAUSS_RTOL)
    assert results[0] == pytest.approx(results[1], rel=GAUSS_RTOL)
    if precision == "fp64":
        # the oracle's residual of the same state (its particles in storage
        # order: electrons and positrons interleaved does not change the sum)
        cell = np.concatenate([parts[0]["cell"], parts[1]["cell"]])
        off = np.concatenate([parts[0]["off"], parts[1]["off"]])
        u = np.concatenate([parts[0]["u"], parts[1]["u"]])
        q = np.concatenate([-np.ones(len(parts[0]["cell"])), np.ones(len(parts[1]["cell"]))]).astype(np.int8)
        r_orc = oracle.Oracle.from_state(_oracle_params(p), cell, off, u, q, E=E_host).diag_now()["gauss_resid"]
        assert r_ref == pytest.approx(r_orc, rel=GAUSS_RTOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_gauss_with_background_charge_and_open_boundaries(precision):
    """The co-rotating frame of Section 7 (rho_GJ in Gauss's law, open
    boundaries) after an outflow has started: particles have departed through
    both boundaries and the field near them has grown.  A perturbed field makes
    the residual O(1); the allocation-free call, cascade_gauss and (FP64) the
    oracle agree on it."""
    p = W.corotating(nx=600, precision=precision, ppc=4)
    (c, o, u, q), E = W.corotating_state(p)
    e, ps = q < 0, q > 0
    st = {"elec": {"cell": c[e], "off": o[e], "u": u[e]}, "posi": {"cell": c[ps], "off": o[ps], "u": u[ps]}, "E": E}
    with Cascade(p, state=st) as run:
        run.step(300)
        parts = [run.particles(s) for s in (0, 1)]
        E_run, _ = run.fields()
    E_host = E_run + np.random.default_rng(7).normal(0.0, 0.3, p["nx"])
    with Cascade(p, state={"elec": parts[0], "posi": parts[1], "E": E_host}) as cas:
        r_ref = cas.gauss()
        d = _device_state(parts, E_host, precision)
        results = [_noalloc(p, parts, d, precision) for _ in range(2)]
    assert r_ref > 0.1
    for r in results:
        assert r == pytest.approx(r_ref, rel=GAUSS_RTOL)
    if precision == "fp64":
        cell = np.concatenate([parts[0]["cell"], parts[1]["cell"]])
        off = np.concatenate([parts[0]["off"], parts[1]["off"]])
        uu = np.concatenate([parts[0]["u"], parts[1]["u"]])
        qq = np.concatenate([-np.ones(len(parts[0]["cell"])), np.ones(len(parts[1]["cell"]))]).astype(np.int8)
        r_orc = oracle.Oracle.from_state(_oracle_params(p), cell, off, uu, qq, E=E_host).diag_now()["gauss_resid"]
        assert r_ref == pytest.approx(r_orc, rel=GAUSS_RTOL)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    E = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(CascadeError) as ei:
        capi.cascade_gauss_noalloc(65537, 0.1, 0.1, capi.CASCADE_FP64, 0, 0, 0, 0, 0, 0, E.data_ptr(), 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    assert "65536" in str(ei.value)
    # a later good call reports no stale message
    assert capi.cascade_gauss_noalloc(8, 0.1, 0.1, capi.CASCADE_FP64, 0, 0, 0, 0, 0, 0, E.data_ptr(), 0) == 0.0
    assert capi.last_error_message() == ""
