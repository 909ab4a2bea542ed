"""The allocation-free Gauss check against the allocating one.

cascade_gauss_noalloc serves callers that cannot allocate device memory
(applications that reserve all device memory for their own pool, plug-ins
whose host program owns every allocation, real-time loops that may not call
cudaMalloc); it keeps its scratch in a static device array instead.  Here it
reads the same state as cascade_gauss, from device buffers the test owns, and
must return the same residual, on two calls in a row (the second call finds
the first one's data in the shared scratch and must clear it).  This file is
collected last so that a stopping run has executed every other test first.
"""
import numpy as np
import pytest

from paper_2012_05587_gb300 import Cascade, CascadeError, capi, workloads as W

pytestmark = pytest.mark.gpu

GAUSS_RTOL = 1e-12  # the FP64 tolerance the Gauss-law tests use


def _state(precision):
    p = dict(W.small_cascade(), precision=precision)
    rng = np.random.default_rng(42)
    # a field that does not satisfy Gauss's law, so the residual is O(1) and
    # both implementations must agree on its value, not just on "small"
    E = p["E0"] + rng.normal(0.0, 0.5, p["nx"])
    return p, E


@pytest.mark.parametrize("precision,dtype_name", [("fp64", "float64"), ("fp32", "float32")])
def test_noalloc_gauss_matches_allocating_entry_point(precision, dtype_name):
    import torch

    p, E0 = _state(precision)
    with Cascade(p) as seed_run:
        seed_run.step(40)  # particles spread over the grid and gain momentum
        parts = [seed_run.particles(s) for s in (0, 1)]
        E_run, _ = seed_run.fields()
    E_host = E_run + (E0 - p["E0"])
    state = {"elec": parts[0], "posi": parts[1], "E": E_host}
    with Cascade(p, state=state) as c:
        r_ref = c.gauss()
        dev = torch.device("cuda", torch.cuda.current_device())
        dt = getattr(torch, dtype_name)
        cell_e = torch.as_tensor(parts[0]["cell"], dtype=torch.int32, device=dev)
        off_e = torch.as_tensor(parts[0]["off"], dtype=dt, device=dev)
        cell_p = torch.as_tensor(parts[1]["cell"], dtype=torch.int32, device=dev)
        off_p = torch.as_tensor(parts[1]["off"], dtype=dt, device=dev)
        E_dev = torch.as_tensor(E_host, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        w = p["n0"] * p["dx"] / p["ppc"]
        prec = capi.CASCADE_FP64 if precision == "fp64" else capi.CASCADE_FP32_MIXED
        torch.cuda.synchronize()
        results = []
        for _ in range(2):
            results.append(capi.cascade_gauss_noalloc(
                p["nx"], p["dx"], w, prec, len(parts[0]["cell"]), cell_e.data_ptr(), off_e.data_ptr(),
                len(parts[1]["cell"]), cell_p.data_ptr(), off_p.data_ptr(), E_dev.data_ptr(), stream))
        assert r_ref > 0.1
        for r in results:
            assert r == pytest.approx(r_ref, rel=GAUSS_RTOL)
        assert results[0] == pytest.approx(results[1], rel=GAUSS_RTOL)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    E = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(CascadeError) as ei:
        capi.cascade_gauss_noalloc(65537, 0.1, 0.1, capi.CASCADE_FP64, 0, 0, 0, 0, 0, 0,
                                   E.data_ptr(), 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    assert "65536" in str(ei.value)
