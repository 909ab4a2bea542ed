"""Batched cascades and admission-driven serving, against the oracle and
against each member run alone."""
import numpy as np
import pytest

import oracle
from paper_2012_05587_gb300 import Cascade, CascadeBatch, CascadeError, capi, workloads as W

import test_gpu_parity as T

pytestmark = pytest.mark.gpu


def members_fp64():
    """Uneven grids and particle counts, in-place and long photon flights."""
    return [
        dict(W.small_cascade(), precision="fp64"),
        dict(nx=300, ppc=3, dx=0.07, dt=0.03, n0=1.0, u_spread=0.05, seed=311, E0=12.0, gamma_thr=20.0,
             eps_gamma=8.0, l_pp=0.37, particle_cap=1 << 16, precision="fp64"),
        dict(nx=97, ppc=5, dx=0.07, dt=0.03, n0=1.0, u_spread=0.05, seed=108, E0=12.0, gamma_thr=20.0,
             eps_gamma=8.0, l_pp=0.0, particle_cap=1 << 16, precision="fp64"),
        dict(nx=1031, ppc=2, dx=0.07, dt=0.03, n0=1.0, u_spread=0.05, seed=1042, E0=12.0, gamma_thr=20.0,
             eps_gamma=8.0, l_pp=2.5, particle_cap=1 << 16, precision="fp64"),
    ]


def test_batch_fp64_members_match_oracle():
    """Every member of an FP64 batch against the oracle, per step, to the
    parity horizon (the batch adds each CTA's current with FP64 atomics, so
    only the summation order differs from the oracle).  These small members
    are split across many CTAs by the cost-balanced partition."""
    ps = members_fp64()
    steps = 300
    with CascadeBatch(ps) as b:
        b.step([steps] * len(ps))
        for i, p in enumerate(ps):
            d = b.diag(i, steps)
            E, J = b.fields(i)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, J_ref = ref.fields()
            hz = T.horizon(d_ref, d)
            assert hz >= 60, (i, hz)
            m = d_ref["step"] < hz
            scale = np.abs(d_ref["E_absmax"][m]).max()
            assert np.abs(d["E_mean"][m] - d_ref["E_mean"][m]).max() <= T.RTOL * scale
            assert np.abs(d["U_K"][m] - d_ref["U_K"][m]).max() <= T.RTOL * np.abs(d_ref["U_K"][m]).max()
            if hz > steps:
                assert np.abs(E - E_ref).max() <= T.RTOL * np.abs(E_ref).max()


def _ens(d):
    return T._ensemble(d)


def test_member_alone_and_in_a_mix_agree():
    """The small cascade (FP32) alone and inside a batch of eight uneven
    cascades: same ensemble diagnostics within 2%, and the same physics as
    the single-cascade path."""
    p = W.small_cascade(precision="fp32")
    others = [dict(q) for q in W.batch_scan(7, steps=0)]
    for q in others:
        q.pop("steps")
    steps = p["steps"]
    with CascadeBatch([p]) as alone:
        alone.step([steps])
        d_alone = alone.diag(0, steps)
    mix = [p] + others
    with CascadeBatch(mix) as b:
        b.step([steps] + [300] * len(others))
        d_mix = b.diag(0, steps)
        for i in range(1, len(mix)):
            assert b.counts(i)["step"] == 300
    with Cascade(p) as c:
        c.step(steps)
        d_single = c.diag(steps)
    e_alone, e_mix, e_single = _ens(d_alone), _ens(d_mix), _ens(d_single)
    for k in ("pairs", "peak_after_screen", "period", "energy", "first_zero"):
        assert e_mix[k] == pytest.approx(e_alone[k], rel=0.02), k
        assert e_single[k] == pytest.approx(e_alone[k], rel=0.02), k
    # before the instability amplifies round-off the trajectories coincide
    assert np.abs(d_mix["E_mean"][:100] - d_alone["E_mean"][:100]).max() <= 1e-3 * 10.0


def test_admission_slots_budget_and_release():
    small = dict(W.small_cascade(precision="fp32"), particle_cap=1 << 16)
    _, need = capi.cascade_footprint(small)
    with CascadeBatch(slots=3, precision="fp32", max_nx=1024, hbm_budget=int(2.5 * need)) as b:
        s0 = b.admit(small, 50)
        s1 = b.admit(dict(small, seed=9), 80)
        with pytest.raises(CascadeError) as ei:  # budget: 2.5 footprints
            b.admit(dict(small, seed=10), 10)
        assert ei.value.status == capi.CASCADE_ERR_BUSY
        with pytest.raises(CascadeError):  # grid beyond the batch's max_nx
            b.admit(dict(small, nx=2048), 10)
        with pytest.raises(CascadeError):  # other precision
            b.admit(dict(small, precision="fp64"), 10)
        done = []
        for _ in range(20):
            b.run(16)
            done += b.poll()
        done += b.poll(wait=True)
        assert sorted(done) == sorted([s0, s1])
        assert b.counts(s0)["step"] == 50 and b.counts(s1)["step"] == 80
        b.release(s0)
        s2 = b.admit(dict(small, seed=10), 30)
        assert s2 == s0
        b.run(40)
        assert b.poll(wait=True) == [s2]
        assert b.info()["occupied"] == 2


def test_served_request_matches_running_alone():
    """A request admitted while others are running gives the same result as
    the request run alone (FP64 members: per-step parity to the horizon)."""
    ps = members_fp64()
    req = ps[0]
    steps = 200
    with CascadeBatch(slots=4, precision="fp64", max_nx=2048) as b:
        b.admit(ps[1], 400)
        b.admit(ps[3], 400)
        b.run(50)
        slot = b.admit(req, steps)
        got = []
        while slot not in got:
            b.run(16)
            got += b.poll()
        d_mix = b.diag(slot, steps)
    with Cascade(req) as c:
        c.step(steps)
        d_alone = c.diag(steps)
    hz = T.horizon(d_alone, d_mix)
    assert hz > 100
    m = d_alone["step"] < hz
    assert np.abs(d_mix["E_mean"][m] - d_alone["E_mean"][m]).max() <= T.RTOL * np.abs(d_alone["E_absmax"]).max()


def test_full_scan_members_match_oracle_first_steps():
    """The benchmark's launch configuration: all 256 cascades of the seeded
    parameter scan in one FP32 batch.  For the first 60 steps, five members
    (the three smallest, the median and the largest) are compared with the
    FP64 oracle running each alone: E and J per edge to 2e-4 of max |E|, and
    the counts within 1%."""
    scan = [dict(q) for q in W.batch_scan(256)]
    for q in scan:
        q.pop("steps")
    steps = 60
    order = sorted(range(len(scan)), key=lambda i: scan[i]["nx"] * scan[i]["ppc"])
    picks = order[:3] + [order[len(order) // 2], order[-1]]
    with CascadeBatch(scan) as b:
        b.step([steps] * len(scan))
        for i in picks:
            p = scan[i]
            d = b.diag(i, steps)
            E, J = b.fields(i)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, J_ref = ref.fields()
            scale = np.abs(E_ref).max()
            assert np.abs(E - E_ref).max() <= 2e-4 * scale, i
            assert np.abs(J - J_ref).max() <= 2e-3 * max(np.abs(J_ref).max(), 1e-12) + 2e-4 * scale, i
            for k in ("n_elec", "n_posi", "n_pairs_total"):
                assert abs(d[k][-1] - d_ref[k][-1]) <= 0.01 * max(d_ref[k][-1], 1), (i, k)
            assert np.allclose(d["E_mean"], d_ref["E_mean"], rtol=0, atol=2e-4 * scale), i


@pytest.mark.parametrize("precision", ["fp32", "fp32_fine"])
def test_fp32_batch_members_match_oracle_first_steps(precision):
    """Both FP32 accumulator forms of the batched particle kernel (one int32
    word per edge, and the two-word fine form) against the FP64 oracle: the
    uneven members of the FP64 test, 80 steps (through the first emissions
    and conversions), E per edge and the per-step mean field to 5e-4 of
    max |E|, pair counts within 2%."""
    ps = [dict(p, precision=precision) for p in members_fp64()]
    steps = 80
    with CascadeBatch(ps) as b:
        b.step([steps] * len(ps))
        for i, p in enumerate(ps):
            d = b.diag(i, steps)
            E, _ = b.fields(i)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, _ = ref.fields()
            scale = np.abs(d_ref["E_absmax"]).max()
            assert np.abs(E - E_ref).max() <= 5e-4 * scale, i
            assert np.abs(d["E_mean"] - d_ref["E_mean"]).max() <= 5e-4 * scale, i
            assert abs(d["n_pairs_total"][-1] - d_ref["n_pairs_total"][-1]) <= 0.02 * max(d_ref["n_pairs_total"][-1], 1)


def test_fp32_request_admitted_mid_run_matches_running_alone():
    """Continuous batching in FP32: a request admitted while two other
    cascades are 50 steps into their runs gives the result it gives alone.
    The batched kernel rounds its fixed-point current at a scale set by each
    CTA's share of the batch, so the member alone and in the mix differ by
    round-off, which the instability of Section 5 amplifies only late: the
    first 100 steps agree to 1e-3 of max |E|, and the ensemble diagnostics
    of the whole run (final pairs, screening time, peak field after
    screening, oscillation period, final energy) to 2%."""
    req = W.small_cascade(precision="fp32")
    steps = req["steps"]
    others = [dict(q, precision="fp32") for q in members_fp64()[1:]]
    with CascadeBatch(slots=4, precision="fp32", max_nx=2048) as b:
        b.admit(others[0], 1200)
        b.admit(others[2], 1200)
        b.run(50)
        slot = b.admit(req, steps)
        got = []
        for _ in range(200):
            b.run(16)
            got += b.poll()
            if slot in got:
                break
        assert slot in got
        d_mix = b.diag(slot, steps)
        assert b.counts(slot)["step"] == steps
    with CascadeBatch([req]) as alone:
        alone.step([steps])
        d_alone = alone.diag(0, steps)
    assert np.abs(d_mix["E_mean"][:100] - d_alone["E_mean"][:100]).max() <= 1e-3 * np.abs(d_alone["E_absmax"]).max()
    e_mix, e_alone = _ens(d_mix), _ens(d_alone)
    for k in ("pairs", "peak_after_screen", "period", "energy", "first_zero"):
        assert e_mix[k] == pytest.approx(e_alone[k], rel=0.02), k


def test_autotuned_scan_matches_oracle_and_caches_its_choice(tmp_path, monkeypatch):
    """Autotuning of the batched particle kernel (the scan's launch shape is
    picked by measurement).  The 256-cascade scan, armed to measure even on a
    cache hit, runs its first steps cycling through every candidate variant
    (five launch shapes, with and without cp.async staging), one step each,
    then continues with the fastest.  Every step was computed by whichever
    variant it drew, so the members' agreement with the FP64 oracle at step
    60 covers all candidates.  The choice is stored under the batch's size
    class, and a second batch of the same class takes it from the cache."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CASCADE_TUNE_CACHE", str(cache))
    scan = [dict(q) for q in W.batch_scan(256)]
    for q in scan:
        q.pop("steps")
    steps = 60
    order = sorted(range(len(scan)), key=lambda i: scan[i]["nx"] * scan[i]["ppc"])
    picks = [order[0], order[len(order) // 2], order[-1]]
    with CascadeBatch(scan) as b:
        b.tune_next(rounds=4, use_cache=False)
        b.step([steps] * len(scan))
        v = b.variant()
        assert v["source"] == "tuned" and v["ns_per_unit"] > 0, v
        for i in picks:
            p = scan[i]
            E, _ = b.fields(i)
            d = b.diag(i, steps)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, _ = ref.fields()
            scale = np.abs(E_ref).max()
            assert np.abs(E - E_ref).max() <= 2e-4 * scale, i
            for k in ("n_elec", "n_posi", "n_pairs_total"):
                assert abs(d[k][-1] - d_ref[k][-1]) <= 0.01 * max(d_ref[k][-1], 1), (i, k)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[1] == f"{v['shape']} {v['stage']} {v['prefetch']} {v['member_cost']}"
    with CascadeBatch(scan) as b2:
        b2.step([16] * len(scan))
        v2 = b2.variant()
        assert v2["source"] == "cached"
        assert (v2["shape"], v2["stage"], v2["prefetch"]) == (v["shape"], v["stage"], v["prefetch"])


def test_forced_variant_and_tuning_off(monkeypatch):
    """A forced variant (the measurement overrides) turns tuning off and is
    used as given; one that does not fit the batch is rejected."""
    p = W.small_cascade(precision="fp32")
    with CascadeBatch([p]) as b:
        b.set_variant(shape=1, stage=0, prefetch=2, member_cost=512)
        b.step([32])
        v = b.variant()
        assert v["source"] == "forced" and (v["shape"], v["stage"], v["prefetch"], v["member_cost"]) == (1, 0, 2, 512)
        with pytest.raises(CascadeError):
            b.set_variant(shape=7, stage=0, prefetch=0)
    monkeypatch.setenv("CASCADE_BATCH_SHAPE", "2")
    with CascadeBatch([p]) as b:
        b.step([32])
        assert b.variant()["source"] == "forced" and b.variant()["shape"] == 2


@pytest.mark.parametrize("precision,stage", [("fp32", 1), ("fp32", 0), ("fp32_fine", 1)])
def test_constant_bank_kernel_matches_oracle(precision, stage):
    """Launch shape 4, the constant-bank form of the batched particle kernel
    (one row of CTAs per member, the member's descriptor read from the
    constant bank by blockIdx.y): the uneven members of the FP64 test in
    FP32, 80 steps through the first emissions and conversions, against the
    FP64 oracle with the tolerances of the persistent kernel's test."""
    ps = [dict(p, precision=precision) for p in members_fp64()]
    steps = 80
    with CascadeBatch(ps) as b:
        b.set_variant(shape=4, stage=stage, prefetch=0 if stage else 1)
        b.step([steps] * len(ps))
        assert b.variant()["shape"] == 4
        for i, p in enumerate(ps):
            d = b.diag(i, steps)
            E, _ = b.fields(i)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, _ = ref.fields()
            scale = np.abs(d_ref["E_absmax"]).max()
            assert np.abs(E - E_ref).max() <= 5e-4 * scale, i
            assert np.abs(d["E_mean"] - d_ref["E_mean"]).max() <= 5e-4 * scale, i
            assert abs(d["n_pairs_total"][-1] - d_ref["n_pairs_total"][-1]) <= 0.02 * max(d_ref["n_pairs_total"][-1], 1)


def test_constant_bank_kernel_on_the_scan_and_mid_run_admission():
    """The constant-bank kernel on all 256 cascades of the scan (first 60
    steps, five members against the oracle), then on a served batch where a
    request joins two running members: the joining member's table entry is
    written behind the queued steps, and its result matches the same request
    run with the persistent kernel (first 100 steps to 1e-3 of max |E|)."""
    scan = [dict(q) for q in W.batch_scan(256)]
    for q in scan:
        q.pop("steps")
    steps = 60
    order = sorted(range(len(scan)), key=lambda i: scan[i]["nx"] * scan[i]["ppc"])
    picks = order[:2] + [order[len(order) // 2], order[-2], order[-1]]
    with CascadeBatch(scan) as b:
        b.set_variant(shape=4, stage=1, prefetch=0)
        b.step([steps] * len(scan))
        for i in picks:
            p = scan[i]
            E, _ = b.fields(i)
            d = b.diag(i, steps)
            ref = oracle.Oracle(T.oracle_params(p))
            d_ref = ref.step(steps)
            E_ref, _ = ref.fields()
            assert np.abs(E - E_ref).max() <= 2e-4 * np.abs(E_ref).max(), i
            for k in ("n_elec", "n_posi", "n_pairs_total"):
                assert abs(d[k][-1] - d_ref[k][-1]) <= 0.01 * max(d_ref[k][-1], 1), (i, k)
    req = W.small_cascade(precision="fp32")
    others = [dict(q, precision="fp32") for q in members_fp64()[1:]]
    out = {}
    for shape, stage in ((4, 1), (3, 1)):
        with CascadeBatch(slots=4, precision="fp32", max_nx=2048) as b:
            b.set_variant(shape=shape, stage=stage, prefetch=0)
            b.admit(others[0], 400)
            b.admit(others[2], 400)
            b.run(50)
            slot = b.admit(req, 100)
            got = []
            for _ in range(200):
                b.run(16)
                got += b.poll()
                if slot in got:
                    break
            assert slot in got
            out[shape] = b.diag(slot, 100)
    scale = np.abs(out[3]["E_absmax"]).max()
    assert np.abs(out[4]["E_mean"] - out[3]["E_mean"]).max() <= 1e-3 * scale
    assert abs(out[4]["n_pairs_total"][-1] - out[3]["n_pairs_total"][-1]) <= 0.01 * out[3]["n_pairs_total"][-1]


def test_member_table_exhaustion_falls_back():
    """The constant bank holds a few hundred member entries per precision: a
    batch that finds no free slice keeps the shared-memory kernel (launch
    shape 4 is refused for it), and the slice returns when its owner goes."""
    a = CascadeBatch(slots=300, precision="fp32", max_nx=1024)
    try:
        a.set_variant(shape=4, stage=1, prefetch=0)
        b = CascadeBatch(slots=300, precision="fp32", max_nx=1024)
        try:
            with pytest.raises(CascadeError):
                b.set_variant(shape=4, stage=1, prefetch=0)
        finally:
            b.close()
    finally:
        a.close()
    with CascadeBatch(slots=300, precision="fp32", max_nx=1024) as c:
        c.set_variant(shape=4, stage=1, prefetch=0)
