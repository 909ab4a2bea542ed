"""Benchmark: particle-steps/s of the large pair cascade on GB300.

Workload (N = 1): the large single cascade -- Nx = 16384, dx = 0.05,
dt = 0.025, 64 e- + 64 e+ per cell, E0 = 100, gamma_thr = 50, eps_gamma = 20,
l_pp = 0.5, FP32-mixed, particle cap 5e8 -- advanced through its cascade and
field screening (``--prep`` steps, untimed) so the timed steps run at full
multiplicity.  One step = one pass of the whole path: photon conversion,
gather/push/move/deposit/emission, Ampere update, diagnostics.

value      particle-steps/s over the K timed steps (device clock, inputs
           resident in HBM; the particle state, several GB, exceeds L2)
e2e        the same metric through the C ABI with host buffers: the state is
           uploaded from pinned host memory, every step's record is read back
           to the host, and the final E/J are read back
roofline   the particle kernel against the measured HBM copy bandwidth:
           24 algorithmic bytes per particle-step (int32 cell + FP32 offset +
           FP32 momentum, read and written)
qed_active the same metric and roofline on two timed phases in which the
           QED model works: the cascade itself (steps 0-200, the particle
           count growing from the seed to screening) and the secondary pair
           bursts that damp the oscillation (from step 1000)
batch_scan the 256-cascade parameter scan for its first 300 steps in one
           batch: its particle-steps/s and the batched particle kernel's
           roofline (``--workload batch`` runs the full 3000 steps)
serving    150 requests of the serving distribution arriving at 5 per second
           (below capacity): aggregate particle-steps/s and p50/p99 time to
           result (``--workload serve`` runs 2000 requests, saturated and
           below capacity)
cpu_baseline  the FP64 oracle on a bounded slice of the same workload

``--impl reference`` times the oracle (the only reference this method has)
on the host cores, on an Nx = 512 slice of the same cascade.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s incl. deposit+QED (batched FP32 vs plain FP64), % HBM roofline; p50/p99"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = {"fp32": 24, "fp64": 40}
# DRAM bytes (read + write) per particle-step of the FP32 particle kernel (the
# form that stages its particles through shared memory): dram__bytes_read.sum +
# dram__bytes_write.sum = 418.6 + 366.7 MB for 3.487e7 particle-steps in one
# launch, from "ncu --set full --clock-control none -k regex:k_push -s 203 -c 2
# python bench.py --steps 10 --warmup 3 --prep 200 --ppc 8 --cap 25000000
# --no-e2e --no-cpu" (a post-screening case of the same grid, 8 + 8 seed
# particles per cell); traffic grows in proportion to the particles processed.
MEASURED_DRAM_BYTES_PER_PARTICLE_STEP = {"fp32": 22.52}
# The FP64 particle kernel is bound by the FP64 pipe, not by HBM: ncu counted
# 45,085,174 FP64-pipe warp instructions for 34,865,152 particle-steps
# (sm__inst_executed_pipe_fp64.sum on the same post-screening case as above,
# with the FP64 pipe busy 84.9% of the cycles and DRAM at 6%).  The pipe's peak is
# 9.5 warp instructions per cycle for the GPU: one per 16 cycles on each of
# the 152 SMs (2 FP64 lanes per SM per cycle, which is 1.26 TFLOP/s of FMA at
# 2.07 GHz); ncu reports the same figure as the metric's peak_sustained.
FP64_PIPE_INST_PER_PARTICLE_STEP = 45_085_174 / 34_865_152
FP64_PIPE_PEAK_INST_PER_CYCLE = 152 / 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prep", type=int, default=400, help="untimed steps that grow the cascade")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cascade-steps", type=int, default=200,
                    help="large workload: first steps timed as the cascade phase (0 = skip)")
    ap.add_argument("--burst-start", type=int, default=1000,
                    help="large workload: step where the timed secondary-burst phase starts (0 = skip)")
    ap.add_argument("--burst-steps", type=int, default=100)
    ap.add_argument("--serve-summary-requests", type=int, default=150,
                    help="large workload: requests of the serving entry (0 = skip)")
    ap.add_argument("--serve-summary-rate", type=float, default=5.0,
                    help="large workload: arrival rate of the serving entry (requests/s)")
    ap.add_argument("--batch-summary-steps", type=int, default=300,
                    help="large workload: steps of the batched scan timed for the batch_scan entry (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cap", type=int, default=0, help="particle cap per species (0 = the workload's)")
    ap.add_argument("--ppc", type=int, default=0, help="seed particles per cell per species (0 = the workload's)")
    ap.add_argument("--u-words", type=int, default=0,
                    help="FP32 momentum words (0 = chosen at creation, 2 = compensated pair: 28 B per particle-step)")
    ap.add_argument("--workload", default="large",
                    choices=["large", "batch", "serve", "sweep", "paper", "corotating", "damping", "parity"],
                    help="large: one large cascade (default); batch: the 256-cascade parameter scan in one "
                         "launch per step; serve: Poisson arrivals admitted by footprint; sweep: FP32 vs FP64 "
                         "errors of the ensemble diagnostics")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=3000)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--serve-low-frac", type=float, default=0.5,
                    help="serve workload: second run at this fraction of the measured capacity (0 = skip)")
    ap.add_argument("--serve-low-requests", type=int, default=400)
    ap.add_argument("--fp64-sample", type=int, default=32,
                    help="cascades run one at a time in FP64 for comparison, spread evenly over the predicted "
                         "particle-steps (0 = none, -1 = every scan member or request)")
    ap.add_argument("--paper-time", type=float, default=12.0, help="paper workload: simulated time (1/omega_p)")
    ap.add_argument("--paper-fs", default="0.1,0.01,0.004", help="paper workload: values of f")
    ap.add_argument("--paper-dt-factors", default="1", help="paper workload: multiples of the paper's time step")
    ap.add_argument("--save-series", default="", help="paper/corotating workloads: directory for the series")
    ap.add_argument("--corot-time", type=float, default=200.0, help="corotating workload: simulated time")
    ap.add_argument("--sweep-seeds", type=int, default=8, help="sweep workload: seeds averaged per configuration")
    ap.add_argument("--damping-seeds", type=int, default=32, help="damping workload: seeds per precision")
    ap.add_argument("--parity-steps", type=int, default=800, help="parity workload: steps of the large cascade")
    ap.add_argument("--sweep-rows", default="", help="sweep workload: comma-separated configuration indices (all)")
    return ap.parse_args()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu() -> str:
    """The host processor as /proc/cpuinfo names it (model name on x86; the
    implementer and part codes on Arm), with the architecture and core count."""
    import platform

    model = None
    fields = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" not in line:
                continue
            k, v = (x.strip() for x in line.split(":", 1))
            if k == "model name" and model is None:
                model = v
            if k in ("CPU implementer", "CPU part") and k not in fields:
                fields[k] = v
    except OSError:
        pass
    if model is None and fields:
        model = ", ".join(f"{k} {v}" for k, v in fields.items())
    return f"{platform.machine()}, {os.cpu_count()} cores, {model or 'unknown model'}"


def oracle_slice(steps_prep: int, steps_timed: int, multicore: bool = False):
    """FP64 oracle on an Nx = 512 slice of the large cascade (same dx, dt,
    ppc, E0, gamma_thr, eps_gamma, l_pp).  Returns particle-steps/s of the
    timed steps, the particle-steps, the seconds, the threads used and what was
    timed.  ``multicore`` runs the OpenMP build of the same source on every
    host core."""
    import oracle
    from paper_2012_05587_gb300 import workloads as W

    p = W.large_cascade(precision="fp64")
    p = {k: v for k, v in p.items() if k not in ("precision", "steps")}
    p["nx"] = 512
    p["particle_cap"] = 1 << 26
    lib = None
    threads = 1
    if multicore:
        lib = oracle.build_multicore()
        threads = os.cpu_count() or 1
        oracle._load(lib).orc_set_threads(threads)
        threads = int(oracle._load(lib).orc_threads())
    o = oracle.Oracle(p, lib_path=lib)
    if steps_prep:
        o.step(steps_prep)
    t0 = time.perf_counter()
    d = o.step(steps_timed)
    el = time.perf_counter() - t0
    ps = float((d["n_elec"] + d["n_posi"]).sum())
    what = "multi-core (OpenMP) build" if multicore else "plain build"
    return ps / el, ps, el, threads, (f"FP64 oracle, {what}, {threads} thread(s), Nx=512 slice of the large cascade "
                                      f"(64+64 per cell), steps {steps_prep}-{steps_prep + steps_timed}, "
                                      f"{ps:.3g} particle-steps in {el:.1f} s")


def aggregate_over_ranks(ms: float, particle_steps: float, device: str = "cuda"):
    """Whole-job figures of N independent replicas: the slowest rank's time and
    the particle-steps of all ranks (no data-path exchange: each rank runs its
    own cascade).  With one rank, the rank's own numbers."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, particle_steps
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    p = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # the oracle as it stands: prep to the post-screening phase, then W + K steps
    import oracle
    from paper_2012_05587_gb300 import workloads as W

    p = W.large_cascade(precision="fp64")
    p = {k: v for k, v in p.items() if k not in ("precision", "steps")}
    p["nx"] = 512
    p["particle_cap"] = 1 << 26
    o = oracle.Oracle(p)
    o.step(args.prep)
    o.step(args.warmup)
    t0 = time.perf_counter()
    d = o.step(args.steps)
    el = time.perf_counter() - t0
    ps = float((d["n_elec"] + d["n_posi"]).sum())
    v = ps / el
    sample = (f"FP64 oracle, 1 thread, Nx=512 slice of the large cascade, steps "
              f"{args.prep + args.warmup}-{args.prep + args.warmup + args.steps}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "large cascade slice Nx=512 (64+64 per cell, E0=100, gamma_thr=50, eps=20, "
                               "l_pp=0.5, dt=0.025, dx=0.05)", "l2": "state fits in host caches; CPU run"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "large":
        import bench_workloads

        return bench_workloads.run(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2012_05587_gb300 import Cascade, capi, workloads as W

    prec = args.precision
    p = W.large_cascade(run=rank, precision=prec)
    if prec == "fp64":
        p["particle_cap"] = 200_000_000  # 3.1e8 particles by step 1200, 20 B each
    if args.cap:
        p["particle_cap"] = args.cap
    if args.ppc:
        p["ppc"] = args.ppc
    if args.u_words:
        p["u_words"] = args.u_words
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    peak, peak_kind = measured_peak()
    bpp = BYTES_PER_PARTICLE_STEP[prec]
    if prec == "fp32" and capi.cascade_momentum_words(p) == 2:
        bpp += 4  # the low word of a two-word momentum, read and written
    c = Cascade(p)
    # the cascade phase, with emission and pair creation at every step
    casc = None
    if args.cascade_steps > 0:
        casc = timed_phase(c, min(args.cascade_steps, args.prep), stream, bpp, peak, prec)
        casc["what"] = (f"steps 0-{casc['steps']}: the pair cascade, from the seed to screening "
                        "(emission, photon flight and pair creation active)")
    c.step(args.prep - (casc["steps"] if casc else 0))
    c.step(args.warmup)
    c.sync()
    capi.cascade_set_timing(c.h, True)
    capi.cascade_timing(c.h)  # clear
    sampler = ClockSampler(torch.cuda.current_device())
    barrier()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    c.step(args.steps)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    tim = capi.cascade_timing(c.h)
    capi.cascade_set_timing(c.h, False)
    rec = c.diag(args.steps)
    c.sync()
    assert len(rec["step"]) == args.steps
    ps = float((rec["n_elec"] + rec["n_posi"]).sum())
    n_now = int(rec["n_elec"][-1] + rec["n_posi"][-1])
    pairs_timed = int(rec["n_pairs_total"][-1] - rec["n_pairs_total"][0])

    t_max, ps_all = aggregate_over_ranks(ms, ps, "cuda")
    value = ps_all / (t_max / 1e3)

    avg_push_s = tim["particle_kernel_ms"] / 1e3 / max(tim["particle_kernel_launches"], 1)
    achieved = bpp * ps / args.steps / avg_push_s / 1e9
    tb = MEASURED_DRAM_BYTES_PER_PARTICLE_STEP.get(prec) if bpp == BYTES_PER_PARTICLE_STEP[prec] else None
    traffic = tb * ps / args.steps if tb else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": "ncu capture of a smaller case scaled per particle-step"
            if tb else None, "kernel": "k_push (gather/push/move/deposit/emission)",
            "bytes_per_particle_step": bpp, "peak_source": peak_kind}
    if prec == "fp64":
        # FP64-pipe bound: warp instructions per second against the pipe's
        # peak at the SM clock sampled during the timed region
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        a = FP64_PIPE_INST_PER_PARTICLE_STEP * ps / args.steps / avg_push_s / 1e9
        pk = FP64_PIPE_PEAK_INST_PER_CYCLE * mhz * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": a, "peak": pk, "unit": "G FP64 warp-inst/s", "frac": a / pk,
                "traffic": None, "kernel": "k_push (gather/push/move/deposit/emission), FP64",
                "inst_per_particle_step": FP64_PIPE_INST_PER_PARTICLE_STEP,
                "peak_source": "152 SMs x 1 FP64 warp instruction per 16 cycles x sampled SM clock",
                "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "bytes_per_particle_step": bpp}}

    # the secondary pair bursts that damp the oscillation (Section 6)
    burst = None
    done = args.prep + args.warmup + args.steps
    if args.burst_start > 0 and args.burst_steps > 0 and args.burst_start >= done:
        c.step(args.burst_start - done)
        burst = timed_phase(c, args.burst_steps, stream, bpp, peak, prec)
        burst["what"] = (f"steps {args.burst_start}-{args.burst_start + args.burst_steps}: secondary pair bursts "
                         "of the damping phase")

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(c, p, args.steps, stream, barrier)
    c.close()

    batch = serving = None
    if prec == "fp32" and args.batch_summary_steps > 0:
        import bench_workloads

        batch = bench_workloads.batch_scan_summary(args.batch_summary_steps)
    if prec == "fp32" and args.serve_summary_requests > 0:
        import bench_workloads

        serving = bench_workloads.serve_summary(args.serve_summary_requests, args.serve_summary_rate)

    cpu = cpu_mc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, psx, el, nt, sample = oracle_slice(150, 60)
        cpu = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample, "host": host_cpu()}
        try:
            v, psx, el, nt, sample = oracle_slice(150, 60, multicore=True)
            cpu_mc = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle (OpenMP build)", "sample": sample,
                      "host": host_cpu()}
        except Exception as e:  # no OpenMP runtime on the host
            cpu_mc = {"unavailable": str(e).splitlines()[0]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": f"large single cascade {prec}: Nx=16384, dx=0.05, dt=0.025, "
                                   f"{p['ppc']}+{p['ppc']} per cell, "
                                   f"E0=100, gamma_thr=50, eps_gamma=20, l_pp=0.5, steps {args.prep + args.warmup}-"
                                   f"{args.prep + args.warmup + args.steps} (post-screening)",
                       "particles_per_step": ps / args.steps, "particles_at_end": n_now,
                       "pairs_created_per_particle_step": pairs_timed / ps,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (particle state >> 129 MB)"},
            "roofline": roof,
            "qed_active": {"cascade_phase": casc, "burst_phase": burst},
            "batch_scan": batch,
            "serving": serving,
            "cpu_baseline": cpu,
            "cpu_multicore": cpu_mc,
            "e2e": e2e,
            "gpu_launches": tim["kernels_launched"] * world,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def timed_phase(c, nsteps, stream, bpp, peak, prec):
    """nsteps steps of a cascade timed on its stream (CUDA events around the
    whole steps and around every particle-kernel launch), with the QED
    activity they contained.  The particle kernel's algorithmic bytes are
    bpp per particle-step plus the photon entries it appends (cell and
    offset: 8 B in FP32, 12 B in FP64)."""
    import torch

    from paper_2012_05587_gb300 import capi

    c.sync()
    capi.cascade_set_timing(c.h, True)
    capi.cascade_timing(c.h)  # clear
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    c.step(nsteps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    tim = capi.cascade_timing(c.h)
    capi.cascade_set_timing(c.h, False)
    rec = c.diag(nsteps)
    ps = float((rec["n_elec"] + rec["n_posi"]).sum())
    pairs = float(rec["n_pairs_total"][-1] - rec["n_pairs_total"][0])
    # photons emitted = photons in flight added + photons converted
    photons = float(rec["n_photon"][-1] - rec["n_photon"][0]) + pairs
    ph_bytes = 8 if prec == "fp32" else 12
    push_s = tim["particle_kernel_ms"] / 1e3
    achieved = (bpp * ps + ph_bytes * photons) / push_s / 1e9 if push_s > 0 else None
    return {"steps": nsteps, "value": ps / (ms / 1e3), "unit": UNIT, "ms": ms,
            "particles_first": int(rec["n_elec"][0] + rec["n_posi"][0]),
            "particles_last": int(rec["n_elec"][-1] + rec["n_posi"][-1]),
            "pairs_created_per_particle_step": pairs / ps, "photons_emitted_per_particle_step": photons / ps,
            "particle_kernel_share": push_s * 1e3 / ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None,
                         "bytes": f"{bpp} B per particle-step + {ph_bytes} B per photon appended"}}


def e2e_run(c, p, steps, stream, barrier):
    """Same workload through the public API with host buffers: upload the
    state from pinned host memory (cascade_create_from_state, FP32 arrays
    for an FP32 cascade), then every step read its record back
    (cascade_diag), finally read E and J.  Closes c."""
    import torch

    from paper_2012_05587_gb300 import Cascade, capi

    cnt = c.counts()
    ne, npo = cnt["n_elec"], cnt["n_posi"]
    E, _ = c.fields()

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    # FP32 cascades take FP32 host arrays (12 B per particle); FP64 ones FP64 (20 B)
    real = torch.float32 if p.get("precision", "fp32") != "fp64" else torch.float64
    host = {}
    for s, n in ((0, ne), (1, npo)):
        part = c.particles(s)
        hc = pinned(n, torch.int32)
        ho = pinned(n, real)
        hu = pinned(n, real)
        hc[:] = part["cell"]
        ho[:] = part["off"]
        hu[:] = part["u"]
        host[s] = {"cell": hc, "off": ho, "u": hu}
    hE = pinned(len(E), torch.float64)
    hE[:] = E
    del part
    # the bench's cascade is released first: its device memory returns to
    # torch's caching allocator, which the new cascade then reuses, as a user
    # running cascades one after another would (a first-ever allocation of the
    # ~6 GB state adds about 60 ms of cudaMalloc to the upload)
    c.close()
    barrier()
    reserved0 = torch.cuda.memory_reserved()
    t0 = time.perf_counter()
    c2 = Cascade(p, state={"elec": host[0], "posi": host[1], "E": hE})
    t_up = time.perf_counter() - t0
    grew = torch.cuda.memory_reserved() - reserved0
    # every step's record reaches the host: queued behind its step, read
    # while the next steps run, the last ones waited for at the end
    ps = 0.0
    got = 0
    for _ in range(steps):
        c2.step(1)
        c2.record_enqueue()
        r = c2.record_poll()
        ps += float((r["n_elec"] + r["n_posi"]).sum())
        got += len(r["step"])
    r = c2.record_poll(wait=True)
    ps += float((r["n_elec"] + r["n_posi"]).sum())
    got += len(r["step"])
    assert got == steps, (got, steps)
    E2, J2 = c2.fields()
    barrier()
    el = time.perf_counter() - t0
    c2.close()
    # the same upload once more (not part of the metric): tells a one-off cost
    # of the first upload from the steady one
    barrier()
    t1 = time.perf_counter()
    c3 = Cascade(p, state={"elec": host[0], "posi": host[1], "E": hE})
    barrier()
    t_again = time.perf_counter() - t1
    c3.close()
    # outside the metric: the same host arrays copied by torch alone, which
    # tells the host memory's copy rate from the library's own upload costs
    barrier()
    t2 = time.perf_counter()
    raw = [torch.from_numpy(host[s][k]).to(stream.device, non_blocking=True) for s in (0, 1)
           for k in ("cell", "off", "u")]
    barrier()
    t_raw = time.perf_counter() - t2
    del raw
    h2d = sum(host[s][k].nbytes for s in (0, 1) for k in ("cell", "off", "u")) + hE.nbytes
    d2h = capi.cascade_record_copy_bytes() * steps + E2.nbytes + J2.nbytes
    return {"value": ps / el, "unit": UNIT, "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": el, "create_and_upload_s": t_up, "steps_and_reads_s": el - t_up,
            "create_and_upload_again_s": t_again, "plain_copy_of_the_host_arrays_s": t_raw,
            "device_memory_reserved_by_the_first_upload_bytes": grew,
            "what": "cascade_create_from_state(_f32) from pinned host arrays (int32 cell, offset and momentum in "
                    "the cascade's precision) + per step cascade_step(1), cascade_record_enqueue and a "
                    "non-blocking cascade_record_poll (every step's record read to the host, the last ones "
                    "waited for) + final E/J to host; wall clock"}


if __name__ == "__main__":
    sys.exit(main())
