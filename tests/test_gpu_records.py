"""Per-step records read while the next steps run (cascade_record_enqueue /
cascade_record_poll): every queued copy arrives, in order, and equals the
record cascade_diag returns for the same step, also when the host queues
more copies than the ring holds in flight."""
import numpy as np
import pytest

from paper_2012_05587_gb300 import Cascade, workloads as W

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


def test_a_full_ring_waits_and_loses_nothing():
    """200 steps queued without a poll: the ring of 64 in-flight copies
    fills, each further enqueue waits for the oldest and keeps it, and one
    poll then returns all 200 records in order."""
    p = dict(W.small_cascade(), precision="fp32")
    with Cascade(p) as c:
        for _ in range(200):
            c.step(1)
            c.record_enqueue()
        r = c.record_poll(max_records=300, wait=True)
        ring = c.diag(200)
    np.testing.assert_array_equal(r["step"], np.arange(1, 201))
    for k in ring:
        np.testing.assert_array_equal(r[k], ring[k], err_msg=k)
