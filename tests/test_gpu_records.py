"""Per-step records read while the next steps run (cascade_record_enqueue /
cascade_record_poll): every queued copy arrives, in order, and equals the
record cascade_diag returns for the same step; a full queue refuses a
further copy without losing any."""
import numpy as np
import pytest

from paper_2012_05587_gb300 import Cascade, CascadeError, capi, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_queued_records_equal_the_ring(precision):
    p = dict(W.small_cascade(), precision=precision)
    steps = 150
    got = []
    with Cascade(p) as c:
        for _ in range(steps):
            c.step(1)
            c.record_enqueue()
            got.append(c.record_poll())
        got.append(c.record_poll(wait=True))
        ring = c.diag(steps)
        assert len(c.record_poll(wait=True)["step"]) == 0  # nothing left
    rec = {k: np.concatenate([g[k] for g in got]) for k in got[0]}
    assert len(rec["step"]) == steps
    np.testing.assert_array_equal(rec["step"], np.arange(1, steps + 1))
    for k in ring:
        np.testing.assert_array_equal(rec[k], ring[k], err_msg=k)


def test_full_queue_is_refused_and_loses_nothing():
    p = dict(W.small_cascade(), precision="fp32")
    with Cascade(p) as c:
        for _ in range(64):
            c.step(1)
            c.record_enqueue()
        c.step(1)
        with pytest.raises(CascadeError) as ei:
            c.record_enqueue()
        assert ei.value.status == capi.CASCADE_ERR_BUSY
        r = c.record_poll(max_records=100, wait=True)
        np.testing.assert_array_equal(r["step"], np.arange(1, 65))
        c.record_enqueue()  # room again
        r = c.record_poll(wait=True)
        np.testing.assert_array_equal(r["step"], [65])
