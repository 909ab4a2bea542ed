"""The batched, served and precision-sweep measurements behind ``bench.py
--workload batch|serve|sweep`` (one JSON line each, same metric and unit as
the large-cascade line)."""
from __future__ import annotations

import json
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


def run_batch(args) -> int:
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, workloads as W

    prec = args.precision
    scan = W.batch_scan(args.batch_n, precision=prec, steps=args.batch_steps)
    stream = torch.cuda.current_stream()
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
    ps = 0.0
    over = 0
    for i in range(len(scan)):
        try:
            ps += _psteps(b.diag(i, args.batch_steps))
        except Exception:
            over += 1
    b.close()
    value = ps / (ms / 1e3)
    fp64 = _fp64_one_at_a_time(scan[: args.fp64_sample], lambda p: args.batch_steps)
    line = {
        "metric": B.METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.batch_steps, "warmup": 0,
        "ms_per_step": ms / args.batch_steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec.startswith("fp32") else "f64", "data": "synthetic",
        "config": {"workload": f"batched parameter scan: {len(scan)} cascades (Nx log-U[256,8192], ppc in "
                               "{8,16,32,64}, E0 and gamma_thr log-U[10,1000], eps = gamma_thr/2, l_pp U[0.2,2]), "
                               f"{args.batch_steps} steps each, {prec}, one launch per kernel per step",
                   "members_over_capacity": over, "create_s": t_create, "wall_s": wall},
        "fp64_one_at_a_time": dict(fp64, per_request_s=None,
                                   sample=f"first {args.fp64_sample} cascades of the scan, each alone in FP64"),
        "batched_over_fp64_one_at_a_time": value / fp64["value"] if fp64["value"] else None,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args) -> int:
    import torch

    from paper_2012_05587_gb300 import CascadeBatch, CascadeError, workloads as W

    prec = args.precision
    reqs = W.serving_requests(args.requests, rate=args.rate, precision=prec)
    free = torch.cuda.mem_get_info()[0]
    budget = int(0.6 * free)
    b = CascadeBatch(slots=256, precision=prec, max_nx=8192, hbm_budget=budget)
    pending = list(reqs)
    queue = []
    slot_req = {}
    done = {}
    ps = 0.0
    t0 = time.perf_counter()
    sampler = B.ClockSampler(torch.cuda.current_device())
    sampler.start()
    busy_rejects = 0
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
            done[id(r)] = (r["arrival"], t_adm, t_done)
            b.release(slot)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    b.close()
    ttr = np.array([d - a for a, _, d in done.values()])
    fp64 = _fp64_one_at_a_time(reqs[: args.fp64_sample], lambda p: p["steps"])
    line = {
        "metric": B.METRIC, "value": ps / wall, "unit": UNIT, "n_gpus": 1, "steps": len(reqs), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec.startswith("fp32") else "f64", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} requests, Poisson arrivals {args.rate}/s, parameters from "
                               "the batch scan, steps U[500,5000], admission by predicted device footprint "
                               f"(budget {budget / 1e9:.1f} GB), continuous batching",
                   "busy_rejections": busy_rejects, "wall_s": wall},
        "p50_time_to_result_s": float(np.percentile(ttr, 50)),
        "p99_time_to_result_s": float(np.percentile(ttr, 99)),
        "fp64_alone": dict(fp64, p50_s=float(np.percentile(fp64["per_request_s"], 50)),
                           p99_s=float(np.percentile(fp64["per_request_s"], 99)), per_request_s=None,
                           sample=f"first {args.fp64_sample} requests, each alone in FP64"),
        "served_over_fp64_alone": (ps / wall) / fp64["value"] if fp64["value"] else None,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args) -> int:
    from paper_2012_05587_gb300 import Cascade, CascadeError, analysis, workloads as W

    rows = []
    for p in W.precision_sweep():
        steps = p["steps"]
        row = {"E0": p["E0"], "gamma_thr": p["gamma_thr"], "dt": p["dt"]}
        res = {}
        for prec in ("fp64", "fp32", "fp32_fine"):
            q = dict(p, precision=prec)
            if prec == "fp64":
                q["particle_cap"] = 120_000_000
            try:
                with Cascade(q) as c:
                    c.step(steps)
                    rec = c.diag(steps)
                res[prec] = analysis.ensemble(rec)
            except CascadeError as e:
                res[prec] = {"error": str(e).split(":")[1].strip() if ":" in str(e) else str(e)}
        row["fp64"] = res["fp64"]
        for prec in ("fp32", "fp32_fine"):
            if "error" in res[prec] or "error" in res["fp64"]:
                row[prec] = res[prec]
            else:
                row[prec + "_rel_err"] = analysis.relative_errors(res[prec], res["fp64"])
        rows.append(row)
        print(json.dumps({"sweep_row": row}), flush=True)
    line = {"metric": B.METRIC, "value": None, "unit": UNIT, "workload": "precision sweep", "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run(args) -> int:
    return {"batch": run_batch, "serve": run_serve, "sweep": run_sweep}[args.workload](args)
