"""Writes tests/golden/damping_oracle.json: ensemble diagnostics of the FP64
oracle on the damping cascade (the f = 0.1 case of Sections 5-6: Nx = 2048,
4 + 4 per cell, E0 = 100, gamma_thr = 50, eps_gamma = 5, in-place pairs,
10000 steps), one entry per seed for runs 0 .. 31.

The values come from the oracle alone (the OpenMP build of
oracle/cascade_oracle.c, all host cores; about 3 minutes per seed on 8
cores) passed through the host-side post-processing the GPU tests apply to
their own records (paper_2012_05587_gb300.analysis: zero crossings, the
envelope's peaks and the fits; no step of the method).  Rerun this script
when the oracle, the workload or those definitions change:

    python tests/golden/make_damping_oracle.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2012_05587_gb300 import analysis as A, workloads as W  # noqa: E402

RUNS = 32


def oracle_params(run: int) -> dict:
    p = W.damping_cascade(run, "fp64")
    return {k: v for k, v in p.items() if k not in ("precision", "steps", "photon_cap", "diag_ring")}


def main():
    lib = oracle.build_multicore()
    oracle._load(lib).orc_set_threads(os.cpu_count() or 1)
    steps = W.damping_cascade(0, "fp64")["steps"]
    out = {"what": __doc__.split("\n\n")[0], "steps": steps, "runs": []}
    for run in range(RUNS):
        p = oracle_params(run)
        t0 = time.time()
        rec = oracle.Oracle(p, lib_path=lib).step(steps)
        e = A.ensemble(rec, dict(p, steps=steps))
        e["run"] = run
        e["seed"] = p["seed"]
        out["runs"].append(e)
        print(f"run {run}: {time.time() - t0:.0f} s", flush=True)
        # written after every seed, so a stopped run keeps what it finished
        with open(os.path.join(HERE, "damping_oracle.json"), "w") as f:
            json.dump(out, f, indent=1, allow_nan=True)


if __name__ == "__main__":
    main()
