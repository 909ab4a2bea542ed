"""The batched, served and precision-sweep measurements behind ``bench.py
--workload batch|serve|sweep`` (one JSON line each, same metric and unit as
the large-cascade line)."""
from __future__ import annotations

import json
import os
import time

import numpy as np

import bench as B

UNIT = B.UNIT


def _psteps(rec) -> float:
    return float((rec["n_elec"] + rec["n_posi"]).sum())


def _fp64_one_at_a_time(params: list, steps_of) -> dict:
    """Run each cascade alone in plain FP64 (single-cascade path), one after
    the other; aggregate particle-steps/s and per-request times."""
    import torch

    from paper_2012_05587_gb300 import Cascade

    ps_total, t_total, times = 0.0, 0.0, []
    if not params:
        return {"value": None, "unit": UNIT, "cascades": 0, "seconds": 0.0, "per_request_s": [0.0]}
    for p in params:
        q = dict(p, precision="fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Cascade(q) as c:
            n = steps_of(p)
            c.step(n)
            rec = c.diag(n)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        ps_total += _psteps(rec)
        t_total += el
        times.append(el)
    return {"value": ps_total / t_total, "unit": UNIT, "cascades": len(params), "seconds": t_total,
            "per_request_s": times}


def stratified(params: list, n: int, key) -> list:
    """n members spread evenly over ``params`` sorted by ``key`` (every size
    class represented); all of them when n < 0 or n >= len(params), none
    when n == 0."""
    if n == 0:
        return []
    if n < 0 or n >= len(params):
        return list(params)
    order = sorted(range(len(params)), key=lambda i: key(params[i]))
    return [params[order[int((k + 0.5) * len(params) / n)]] for k in range(n)]


def shard_by_work(costs: list, world: int) -> list:
    """Independent cascades over ``world`` GPUs by predicted work: the
    largest first, each to the rank with the least work so far (ties to the
    lower rank), so every rank computes the same assignment without any
    exchange.  Returns each rank's member indices in their original order."""
    if world < 1:
        raise ValueError("world must be at least 1")
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(x) for x in out]


def route_requests(costs: list, world: int) -> list:
    """Requests in arrival order to ``world`` GPUs: each to the rank whose
    requests so far add up to the least predicted work (ties to the lower
    rank).  Deterministic, so every rank routes the same trace alike.
    Returns the rank of each request."""
    if world < 1:
        raise ValueError("world must be at least 1")
    load = [0.0] * world
    out = []
    for c in costs:
        r = min(range(world), key=lambda r: (load[r], r))
        out.append(r)
        load[r] += float(c)
    return out


def merge_served(parts: list) -> dict:
    """Whole-job serving figures from the ranks' own: the particle-steps of
    all ranks over the slowest rank's wall time, and percentiles over every
    request's times (each part holds its requests' times to result and waits
    for admission)."""
    ps = sum(x["particle_steps"] for x in parts)
    wall = max(x["wall_s"] for x in parts)
    ttr = np.concatenate([np.asarray(x["ttr"], float) for x in parts])
    wait = np.concatenate([np.asarray(x["wait"], float) for x in parts])
    n = int(sum(x["requests"] for x in parts))
    return {"particle_steps": ps, "wall_s": wall, "value": ps / wall if wall > 0 else None, "requests": n,
            "p50_time_to_result_s": float(np.percentile(ttr, 50)) if len(ttr) else None,
            "p99_time_to_result_s": float(np.percentile(ttr, 99)) if len(ttr) else None,
            "p50_wait_for_admission_s": float(np.percentile(wait, 50)) if len(wait) else None,
            "p99_wait_for_admission_s": float(np.percentile(wait, 99)) if len(wait) else None,
            "busy_rejections": int(sum(x["busy_rejections"] for x in parts)),
            "requests_per_s": n / wall if wall > 0 else None, "ranks": len(parts)}


def _ranks():
    """(rank, world) of a torchrun launch, with this rank's GPU selected and
    the process group up when there are several; (0, 1) otherwise."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world


def _gather(obj, world: int) -> list:
    import torch.distributed as dist

    if world == 1:
        return [obj]
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out


def _sample_note(n_sample: int, n_all: int, what: str) -> str:
    if n_sample == 0:
        return f"not run (none of the {n_all} {what})"
    if n_sample >= n_all:
        return f"all {n_all} {what}, each alone in FP64"
    return (f"{n_sample} of {n_all} {what}, spread evenly over the predicted particle-steps "
            "(stratified), each alone in FP64")


def run_batch(args) -> int:
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, capi, workloads as W

    prec = args.precision
    rank, world = _ranks()
    full = W.batch_scan(args.batch_n, precision=prec, steps=args.batch_steps)
    # several GPUs: each runs its share of the scan, balanced by predicted work
    mine = shard_by_work([W.predicted_particles(p) for p in full], world)[rank]
    scan = [full[i] for i in mine]
    footprint = sum(capi.cascade_footprint(p)[1] for p in scan)
    predicted = sum(W.predicted_particles(p) for p in scan)
    stream = torch.cuda.current_stream()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = CascadeBatch(scan)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = B.ClockSampler(torch.cuda.current_device())
    sampler.start()
    w0 = time.perf_counter()
    ev0.record(stream)
    b.step([args.batch_steps] * len(scan))
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    variant = b.variant()
    tuning = b.tuning_report()
    ps = 0.0
    over = 0
    pairs = photons = 0
    for i in range(len(scan)):
        try:
            d = b.diag(i, args.batch_steps)
        except Exception:
            over += 1
            continue
        ps += _psteps(d)
        pairs += int(d["n_pairs_total"][-1])
        photons += int(d["n_pairs_total"][-1] + d["n_photon"][-1])
    b.close()
    roof = _batch_roofline(scan, args.batch_steps, prec)
    ms, ps = B.aggregate_over_ranks(ms, ps)
    pairs = int(sum(_gather(pairs, world)))
    photons = int(sum(_gather(photons, world)))
    over = int(sum(_gather(over, world)))
    value = ps / (ms / 1e3)
    if rank != 0:
        return 0
    if world > 1:
        footprint = sum(capi.cascade_footprint(p)[1] for p in full)
        predicted = sum(W.predicted_particles(p) for p in full)
    sample = stratified(full, args.fp64_sample, lambda p: W.predicted_particles(p))
    fp64 = _fp64_one_at_a_time(sample, lambda p: args.batch_steps)
    line = {
        "metric": B.METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.batch_steps,
        "warmup": 0, "ms_per_step": ms / args.batch_steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32" if prec.startswith("fp32") else "f64", "data": "synthetic",
        "config": {"workload": f"batched parameter scan: {len(full)} cascades (Nx log-U[256,8192], ppc in "
                               "{8,16,32,64}, E0 and gamma_thr log-U[10,1000], eps = gamma_thr/2, l_pp U[0.2,2]), "
                               f"{args.batch_steps} steps each, {prec}, one launch per kernel per step",
                   "parallelism": (f"{world} GPUs, the scan's cascades shared by predicted work, one batch "
                                   "per GPU, no data-path exchange") if world > 1 else "single GPU",
                   "members_over_capacity": over, "create_s": t_create, "wall_s": wall,
                   "device_footprint_bytes": footprint, "predicted_particles_at_screening": predicted,
                   "pairs_created_per_particle_step": pairs / ps if ps else None,
                   "photons_emitted_per_particle_step": photons / ps if ps else None},
        "fp64_one_at_a_time": dict(fp64, per_request_s=None,
                                   sample=_sample_note(len(sample), len(scan), "cascades of the scan")),
        "batched_over_fp64_one_at_a_time": value / fp64["value"] if fp64["value"] else None,
        "roofline": roof,
        "variant": variant,
        "tuning": tuning,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_scan_summary(steps: int = 300, n: int = 256, prec: str = "fp32") -> dict:
    """A short run of the batched scan for the default bench line: the n
    cascades of the parameter scan for the first `steps` steps (the cascade
    phase of most members), launched step by step with CUDA events around
    every launch of the batched particle kernel, with the default launch
    variant.  Particle-steps/s over the whole steps and the particle kernel's
    roofline (24 B per particle-step in FP32)."""
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, capi, workloads as W

    scan = W.batch_scan(n, precision=prec, steps=steps)
    peak, peak_kind = B.measured_peak()
    bpp = B.BYTES_PER_PARTICLE_STEP["fp64" if prec == "fp64" else "fp32"]
    stream = torch.cuda.current_stream()
    b = CascadeBatch(scan)
    # the default launch variant, no tuning pass: 300 steps are the growth
    # phase of most members, which would tune for the wrong state and store
    # that choice under the full scan's size class (on the full scan the
    # tuner picks the default variant, the constant-bank kernel, staged)
    b.tune_next(rounds=0)
    capi.cascade_batch_set_timing(b.b, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step([steps] * len(scan))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    tim = capi.cascade_batch_timing(b.b)
    variant = b.variant()
    ps = sum(_psteps(b.diag(i, steps)) for i in range(len(scan)))
    b.close()
    push_s = tim["particle_kernel_ms"] / 1e3
    achieved = bpp * ps / push_s / 1e9
    return {"workload": f"batched parameter scan, {len(scan)} cascades, steps 0-{steps}, {prec}",
            "value": ps / (ms / 1e3), "unit": UNIT, "particle_steps": ps, "ms": ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "k_batch_push", "bytes_per_particle_step": bpp, "peak_source": peak_kind,
                         "particle_kernel_share": push_s * 1e3 / ms},
            "variant": variant, "kernels_launched": tim["kernels_launched"]}


def serve_summary(requests: int = 150, rate: float = 5.0, prec: str = "fp32") -> dict:
    """A short serving run for the default bench line: `requests` requests
    of the serving distribution (batch-scan parameters, steps U[500, 5000])
    arriving as a Poisson stream at `rate` per second -- about a third of
    the capacity measured with the full serving workload, so the times to
    result measure latency rather than queueing -- admitted by footprint and
    run by continuous batching on a private stream."""
    import torch

    from paper_2012_05587_gb300 import workloads as W

    reqs = W.serving_requests(requests, rate=rate, run=2, precision=prec)
    budget = int(0.6 * torch.cuda.mem_get_info()[0])
    prev = torch.cuda.current_stream()
    torch.cuda.set_stream(torch.cuda.Stream())
    try:
        out = _serve(reqs, prec, budget)
    finally:
        torch.cuda.set_stream(prev)
    out.pop("ttr", None)
    out.pop("wait", None)
    out["workload"] = (f"serving: {requests} requests of the serving distribution, Poisson arrivals at {rate}/s, "
                       "admission by predicted device footprint, continuous batching")
    out["unit"] = UNIT
    return out


def _batch_roofline(scan: list, steps: int, prec: str) -> dict:
    """The same scan again, launched step by step with CUDA events around
    every launch of the batched particle kernel: its algorithmic traffic
    (24 B per particle-step in FP32, 40 B in FP64) over its summed duration,
    against the measured HBM copy bandwidth."""
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, capi

    peak, peak_kind = B.measured_peak()
    bpp = B.BYTES_PER_PARTICLE_STEP["fp64" if prec == "fp64" else "fp32"]
    b = CascadeBatch(scan)
    capi.cascade_batch_set_timing(b.b, True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step([steps] * len(scan))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    tim = capi.cascade_batch_timing(b.b)
    ps = 0.0
    for i in range(len(scan)):
        try:
            ps += _psteps(b.diag(i, steps))
        except Exception:
            continue
    b.close()
    push_s = tim["particle_kernel_ms"] / 1e3
    achieved = bpp * ps / push_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_batch_push (gather/push/move/deposit/emission of every member)",
            "bytes_per_particle_step": bpp, "peak_source": peak_kind,
            "particle_kernel_share": push_s * 1e3 / ms, "launches": tim["particle_kernel_launches"],
            "value_with_direct_launches": ps / (ms / 1e3)}


def _serve(reqs: list, prec: str, budget: int) -> dict:
    """Serve ``reqs`` (each with an arrival time) by continuous batching:
    requests are admitted into free slots while their predicted device
    footprint fits the budget, every loop runs 16 batch steps, and finished
    requests are read back and released.  Returns the particle-steps served,
    the wall time and each request's (arrival, admission, result) times."""
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, CascadeError

    b = CascadeBatch(slots=256, precision=prec, max_nx=8192, hbm_budget=budget)
    pending = list(reqs)
    queue = []
    slot_req = {}
    done = []
    ps = 0.0
    busy_rejects = 0
    t0 = time.perf_counter()
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival"] <= now:
            queue.append(pending.pop(0))
        while queue:
            r = queue[0]
            try:
                slot = b.admit(r, r["steps"])
            except CascadeError as e:
                if e.status == -8:  # busy: wait for a slot or memory
                    busy_rejects += 1
                    break
                raise
            slot_req[slot] = (r, time.perf_counter() - t0)
            queue.pop(0)
        if slot_req:
            b.run(16)
            finished = b.poll()
        else:
            finished = []
            if pending:
                time.sleep(max(0.0, min(0.01, pending[0]["arrival"] - now)))
        for slot in finished:
            r, t_adm = slot_req.pop(slot)
            rec = b.diag(slot, r["steps"])
            t_done = time.perf_counter() - t0
            ps += _psteps(rec)
            done.append((r["arrival"], t_adm, t_done))
            b.release(slot)
    wall = time.perf_counter() - t0
    b.close()
    torch.cuda.synchronize()
    ttr = np.array([d - a for a, _, d in done])
    wait = np.array([m - a for a, m, _ in done])
    return {"particle_steps": ps, "wall_s": wall, "value": ps / wall, "requests": len(reqs),
            "p50_time_to_result_s": float(np.percentile(ttr, 50)),
            "p99_time_to_result_s": float(np.percentile(ttr, 99)),
            "p50_wait_for_admission_s": float(np.percentile(wait, 50)),
            "p99_wait_for_admission_s": float(np.percentile(wait, 99)),
            "busy_rejections": busy_rejects, "requests_per_s": len(reqs) / wall,
            "ttr": ttr.tolist(), "wait": wait.tolist()}


def run_serve(args) -> int:
    import torch

    from paper_2012_05587_gb300 import workloads as W

    prec = args.precision
    rank, world = _ranks()
    reqs_all = W.serving_requests(args.requests, rate=args.rate, precision=prec)
    # several GPUs: one server per GPU, each request routed on arrival to the
    # GPU with the least predicted work routed to it so far
    route = route_requests([W.predicted_particles(r) * r["steps"] for r in reqs_all], world)
    reqs = [r for r, k in zip(reqs_all, route) if k == rank]
    free = torch.cuda.mem_get_info()[0]
    budget = int(0.6 * free)
    # a private stream: host reads of finished requests never wait for the batch
    serve_stream = torch.cuda.Stream()
    torch.cuda.set_stream(serve_stream)
    sampler = B.ClockSampler(torch.cuda.current_device())
    sampler.start()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    sat = merge_served(_gather(_serve(reqs, prec, budget), world))
    clocks = sampler.stop()
    # the same request distribution at a fraction of the capacity just
    # measured (requests completed per second while saturated), so that the
    # times to result measure latency rather than queueing
    low = None
    if args.serve_low_frac > 0 and args.serve_low_requests > 0:
        rate = args.serve_low_frac * sat["requests_per_s"]
        low_all = W.serving_requests(args.serve_low_requests, rate=rate, run=1, precision=prec)
        route_low = route_requests([W.predicted_particles(r) * r["steps"] for r in low_all], world)
        reqs_low = [r for r, k in zip(low_all, route_low) if k == rank]
        low = merge_served(_gather(_serve(reqs_low, prec, budget), world))
        low["arrival_rate_per_s"] = rate
        low.pop("ttr", None)
        low.pop("wait", None)
        low["what"] = (f"{len(low_all)} requests of the same distribution (another seed) arriving at "
                       f"{args.serve_low_frac} of the capacity measured by the saturated run")
    if rank != 0:
        return 0
    sample = stratified(reqs_all, args.fp64_sample, lambda p: W.predicted_particles(p) * p["steps"])
    fp64 = _fp64_one_at_a_time(sample, lambda p: p["steps"])
    reqs = reqs_all
    line = {
        "metric": B.METRIC, "value": sat["value"], "unit": UNIT, "n_gpus": world, "steps": len(reqs), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec.startswith("fp32") else "f64", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} requests, Poisson arrivals {args.rate}/s, parameters from "
                               "the batch scan, steps U[500,5000], admission by predicted device footprint "
                               f"(budget {budget / 1e9:.1f} GB), continuous batching",
                   "parallelism": (f"{world} GPUs, one server each, requests routed by predicted work"
                                   if world > 1 else "single GPU"),
                   "busy_rejections": sat["busy_rejections"], "wall_s": sat["wall_s"]},
        "p50_time_to_result_s": sat["p50_time_to_result_s"],
        "p99_time_to_result_s": sat["p99_time_to_result_s"],
        "saturated": {k: v for k, v in sat.items() if k not in ("ttr", "wait")},
        "below_capacity": low,
        "fp64_alone": dict(fp64, p50_s=float(np.percentile(fp64["per_request_s"], 50)) if sample else None,
                           p99_s=float(np.percentile(fp64["per_request_s"], 99)) if sample else None,
                           per_request_s=None, sample=_sample_note(len(sample), len(reqs), "requests")),
        "served_over_fp64_alone": sat["value"] / fp64["value"] if fp64["value"] else None,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args) -> int:
    """Precision sweep: for each (E0, gamma_thr) the ensemble diagnostics of
    FP32-mixed and FP32-mixed-fine runs, averaged over seeds, against the same
    average of all-FP64 runs (relative errors per diagnostic).  A configuration
    whose predicted particle count exceeds the capacity runs one seed only, to
    show the capacity error it returns."""
    from paper_2012_05587_gb300 import Cascade, CascadeError, analysis, workloads as W

    rows = []
    n_cfg = len(W.precision_sweep(run=0))
    which = [int(x) for x in args.sweep_rows.split(",")] if args.sweep_rows else list(range(n_cfg))
    for idx in which:
        t_row = time.perf_counter()
        p0 = W.precision_sweep(run=0)[idx]
        predicted = W.predicted_particles(p0)
        over = predicted > 2 * p0["particle_cap"]
        seeds = [0] if over else list(range(args.sweep_seeds))
        res = {"fp64": [], "fp32": [], "fp32_fine": []}
        counts = {k: [] for k in res}
        errs = {}
        for run in seeds:
            p = W.precision_sweep(run=run)[idx]
            for prec in res:
                q = dict(p, precision=prec)
                if prec == "fp64":
                    q["particle_cap"] = 120_000_000
                try:
                    with Cascade(q) as c:
                        c.step(p["steps"])
                        rec = c.diag(p["steps"])
                    res[prec].append(analysis.ensemble(rec, q))
                    counts[prec].append({k: rec[k] for k in ("t", "n_elec", "n_posi")})
                except CascadeError as e:
                    errs[prec] = str(e).split(":")[1].strip() if ":" in str(e) else str(e)
        row = {"E0": p0["E0"], "gamma_thr": p0["gamma_thr"], "dt": p0["dt"], "seeds": len(seeds),
               "predicted_particles": predicted}
        if errs:
            row["errors"] = errs
        else:
            mean = {k: {f: float(np.nanmean([r[f] for r in v])) for f in v[0]} for k, v in res.items()}
            # the growth rate of the seed average of ln N, between counts fixed
            # by the parameters (the same window for every precision)
            win = analysis.growth_window(p0)
            for k in mean:
                mean[k]["growth_rate"] = analysis.seed_averaged_growth_rate(counts[k], win)
            row["growth_window"] = list(win) if win else None
            row["fp64_mean"] = mean["fp64"]
            row["fp32_rel_err"] = analysis.relative_errors(mean["fp32"], mean["fp64"])
            row["fp32_fine_rel_err"] = analysis.relative_errors(mean["fp32_fine"], mean["fp64"])
            # seed by seed: the signed relative difference of the means and its
            # standard error, which tells a bias from the chaotic spread
            for k in ("fp32", "fp32_fine"):
                pc = analysis.paired_comparison(res[k], res["fp64"])
                row[k + "_paired"] = {f: [v["rel_err"], v["rel_se"]] for f, v in pc.items()}
        row["seconds"] = time.perf_counter() - t_row
        rows.append(row)
        print(json.dumps({"sweep_row": row}), flush=True)
    line = {"metric": B.METRIC, "value": None, "unit": UNIT, "workload": "precision sweep", "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_parity(args) -> int:
    """The benchmark's own state in three precisions: the large cascade
    (Nx = 16384, 64 + 64 per cell) through the cascade, screening and the
    oscillation after it (--parity-steps, 800 by default: six periods) in
    FP32-mixed, FP32-mixed-fine and FP64 on the GPU; per-cell ensemble
    diagnostics of each and the relative error of the FP32 forms against
    FP64.  (The comparison with the FP64 oracle, on a slice of the same
    plasma, is tests/test_gpu_full_size.py.)"""
    import torch

    from paper_2012_05587_gb300 import Cascade, analysis as A, workloads as W

    steps = args.parity_steps
    out = {}
    secs = {}
    for prec in ("fp32", "fp32_fine", "fp64"):
        p = W.large_cascade(precision=prec)
        if prec == "fp64":
            p["particle_cap"] = 200_000_000
        p["diag_ring"] = max(4096, steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Cascade(p) as c:
            c.step(steps)
            rec = c.diag(steps)
        torch.cuda.synchronize()
        secs[prec] = time.perf_counter() - t0
        e = A.ensemble(rec, p)
        e["particles_per_cell"] = float((rec["n_elec"] + rec["n_posi"])[-1]) / p["nx"]
        e["energy_per_cell"] = e.pop("final_energy") / p["nx"]
        e["pairs_per_cell"] = e.pop("final_pairs") / p["nx"]
        out[prec] = e
    line = {"metric": B.METRIC, "value": None, "unit": UNIT,
            "workload": f"large cascade (Nx = 16384, 64 + 64 per cell) for {steps} steps in three precisions",
            "diagnostics": out, "seconds": secs,
            "fp32_rel_err": A.relative_errors(out["fp32"], out["fp64"]),
            "fp32_fine_rel_err": A.relative_errors(out["fp32_fine"], out["fp64"])}
    print(json.dumps(line), flush=True)
    return 0


def run_damping(args) -> int:
    """Damping of the large-amplitude oscillation (Sections 5-6, Eq. 24):
    the f = 0.1 cascade of workloads.damping_cascade over --damping-seeds
    seeds in FP32-mixed, FP32-mixed-fine and FP64.  Reports per ensemble
    diagnostic the FP64 mean and the relative error of each FP32 form with
    its standard error from the seed-by-seed differences."""
    import torch

    from paper_2012_05587_gb300 import Cascade, analysis as A, workloads as W

    t0 = time.perf_counter()
    res = {"fp32": [], "fp32_fine": [], "fp64": []}
    ps = {k: 0.0 for k in res}
    secs = {k: 0.0 for k in res}
    for run in range(args.damping_seeds):
        for prec in res:
            p = W.damping_cascade(run=run, precision=prec)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            with Cascade(p) as c:
                c.step(p["steps"])
                rec = c.diag(p["steps"])
            torch.cuda.synchronize()
            secs[prec] += time.perf_counter() - t1
            ps[prec] += _psteps(rec)
            res[prec].append(A.ensemble(rec, p))
    keys = ("growth_rate", "screening_time", "peak_field_after_screening", "oscillation_frequency", "damping_rate",
            "damping_eps0", "final_pairs", "final_energy")
    p0 = W.damping_cascade()
    line = {"metric": B.METRIC, "value": ps["fp32"] / secs["fp32"], "unit": UNIT,
            "workload": f"damping cascade (f = 0.1, Nx = {p0['nx']}, {p0['steps']} steps), "
                        f"{args.damping_seeds} seeds per precision",
            "fp64_value": ps["fp64"] / secs["fp64"],
            "fp32_vs_fp64": A.paired_comparison(res["fp32"], res["fp64"], keys),
            "fp32_fine_vs_fp64": A.paired_comparison(res["fp32_fine"], res["fp64"], keys),
            "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


def run_paper(args) -> int:
    """The paper-scale cascades of Section 3 (f = 0.1, 0.01, 0.004) against
    Eq. 3 (growth), Eq. 5 (density at screening), Eq. 10 (mean gamma) and
    Eq. 12 (oscillation frequency, with the measured n and <1/gamma^3>)."""
    import torch

    from paper_2012_05587_gb300 import Cascade, analysis as A, workloads as W

    rows = []
    fs = [float(x) for x in args.paper_fs.split(",")]
    factors = [float(x) for x in args.paper_dt_factors.split(",")]
    for f, fac in [(f, fac) for f in fs for fac in factors]:
        p = W.paper_scale(f, args.precision, dt_factor=fac)
        g, eps, E0 = p["gamma_thr"], p["eps_gamma"], p["E0"]
        ta = g / E0
        steps = int(args.paper_time / p["dt"])
        t0 = time.perf_counter()
        with Cascade(p) as c:
            # run to the first zero of <E> (screening), in chunks of a fixed
            # simulated time (0.016, 50 steps at the paper's dt), so that the
            # distribution below is sampled at the same time after screening
            # whatever the time step
            chunk = max(1, int(round(0.016 / p["dt"])))
            done = 0
            recs = []
            while done < steps:
                c.step(chunk)
                done += chunk
                r = c.diag(chunk)
                recs.append(r)
                if (r["E_mean"] <= 0).any():
                    break
            cat = {k: np.concatenate([x[k] for x in recs]) for k in recs[0]}
            st_e, st_p = c.particles(0), c.particles(1)
            u = np.concatenate([st_e["u"], st_p["u"]])
            gam = np.sqrt(1.0 + u * u)
            n_now = len(u) / (2 * p["nx"] * p["ppc"])
            osc_pred = float(np.sqrt(2 * n_now * np.mean(1.0 / gam ** 3)))
            # continue through the oscillations
            c.step(steps - done)
            r2 = c.diag(steps - done)
            full = {k: np.concatenate([cat[k], r2[k]]) for k in cat}
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        t = full["t"]
        N = full["n_elec"] + full["n_posi"]
        z = A.zero_crossings(t, full["E_mean"])
        ts = float(z[0]) if len(z) else float("nan")
        k_s = int(np.searchsorted(t, ts))
        # growth: N between 10x the seed and a tenth of its value at screening
        # growth: fit of ln N over the cascade, from 100x the seed to a third
        # of the count at screening (the cold seed grows in generations, so
        # the fit spans several of them)
        lnN = np.log(N.astype(float))
        m = (N >= 100 * N[0]) & (N <= N[k_s] / 3.0) & (t < ts)
        G = float(np.polyfit(t[m], lnN[m], 1)[0]) if m.sum() > 5 else float("nan")
        if args.save_series:
            np.savez_compressed(os.path.join(args.save_series, f"paper_f{f}.npz"), t=t, N=N, E=full["E_mean"],
                                UK=full["U_K"], UE=full["U_E"], pairs=full["n_pairs_total"])
        ns = full["n_elec"][k_s] / (p["nx"] * p["ppc"])
        L = p["nx"] * p["dx"]
        row = {
            "f": f, "dt": p["dt"], "dt_factor": fac, "steps": steps, "seconds": el,
            "particle_steps": float(N.sum()),
            "growth_rate_t_a": G * ta,
            "eq3_W_2_over_f": A.lambert_growth_rate(E0, g, eps) * ta,
            "renewal_t_a": A.renewal_growth_rate(E0, g, eps) * ta,
            "screening_time": ts,
            "n_s_over_n0": float(ns),
            "eq5_over_measured": float(A.screening_density(E0, g, eps) / ns),
            "kinetic_share_at_screening": float((full["U_K"][k_s] - full["U_K"][0]) / (0.5 * E0 ** 2 * L)),
            "mean_gamma_at_screening": float(gam.mean()),
            "eq10_mean_gamma": float(A.mean_gamma(g, eps)),
            "osc_freq_measured": float(np.pi / np.mean(np.diff(z[:6]))) if len(z) > 3 else float("nan"),
            "eq12_with_measured_n_and_inv_gamma3": osc_pred,
            "final_pairs": float(full["n_pairs_total"][-1]),
            "mean_E_envelope_last_over_first": float(np.abs(full["E_mean"][t > ts]).max() and
                                                     np.abs(full["E_mean"][-len(t) // 10:]).max() /
                                                     np.abs(full["E_mean"][t > ts]).max()),
        }
        rows.append(row)
        print(json.dumps({"paper_row": row}), flush=True)
    print(json.dumps({"metric": B.METRIC, "value": None, "unit": UNIT, "workload": "paper-scale cascades",
                      "rows": rows}), flush=True)
    return 0


def run_corotating(args) -> int:
    """Section 7 at the paper's parameters (L = 1000, dx = 0.1, dt = 1e-3,
    gamma_thr = 5000, f = 0.01, open boundaries, j_m = -1.5 rho_GJ): time to
    the first pairs, pair count, peak gap field, particle-steps/s; optionally
    a space-time map of E every 100 steps (the quantity of Fig. 4a)."""
    import torch

    from paper_2012_05587_gb300 import Cascade, workloads as W

    p = W.corotating(precision=args.precision)
    state, E = W.corotating_state(p)
    c, o, u, q = state
    e, ps_ = q < 0, q > 0
    st = {"elec": {"cell": c[e], "off": o[e], "u": u[e]}, "posi": {"cell": c[ps_], "off": o[ps_], "u": u[ps_]},
          "E": E}
    steps = int(args.corot_time / p["dt"])
    chunk = 100
    snaps, recs = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with Cascade(p, state=st) as cas:
        done = 0
        while done < steps:
            cas.step(chunk)
            done += chunk
            recs.append(cas.diag(chunk))
            if args.save_series:
                snaps.append(cas.fields()[0].astype(np.float32))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    rec = {k: np.concatenate([r[k] for r in recs]) for k in recs[0]}
    pairs = rec["n_pairs_total"]
    first = float(rec["t"][np.argmax(pairs > 0)]) if pairs[-1] > 0 else float("nan")
    if args.save_series:
        np.savez_compressed(os.path.join(args.save_series, "corotating.npz"), t=rec["t"], pairs=pairs,
                            n_elec=rec["n_elec"], n_posi=rec["n_posi"], E_absmax=rec["E_absmax"],
                            E_map=np.array(snaps), dt_map=p["dt"] * chunk)
    line = {"metric": B.METRIC, "value": float((rec["n_elec"] + rec["n_posi"]).sum() / el), "unit": UNIT,
            "workload": "co-rotating frame, Section 7 parameters", "steps": steps, "seconds": el,
            "time_of_first_pairs": first, "pairs_total": int(pairs[-1]), "peak_field": float(rec["E_absmax"].max()),
            "particles_end": int(rec["n_elec"][-1] + rec["n_posi"][-1])}
    print(json.dumps(line), flush=True)
    return 0


def run(args) -> int:
    return {"batch": run_batch, "serve": run_serve, "sweep": run_sweep, "paper": run_paper,
            "corotating": run_corotating, "damping": run_damping, "parity": run_parity}[args.workload](args)
