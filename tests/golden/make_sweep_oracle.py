"""Writes tests/golden/sweep_oracle.json: ensemble diagnostics of the FP64
oracle on the precision sweep's rows that cascade, at Nx = 512 (a slice of
the sweep's Nx = 4096 grid with the same dx, dt, seed density and seeds),
8 seeds each, 5000 steps.

The values come from the oracle alone (the OpenMP build of
oracle/cascade_oracle.c, all host cores) passed through the same host-side
post-processing the GPU tests apply to their own records
(paper_2012_05587_gb300.analysis: zero crossings, peaks and fits of the
per-step records; no step of the method).  Rerun this script when the
oracle or those definitions change:

    python tests/golden/make_sweep_oracle.py
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

ROWS = (0, 3, 4, 8)   # (E0, gamma_thr) = (10, 20), (100, 20), (100, 200), (1000, 2000)
SEEDS = 8
NX = 512
STEPS = 5000


def slice_params(idx: int, run: int) -> dict:
    p = W.precision_sweep(run=run)[idx]
    p = {k: v for k, v in p.items() if k not in ("precision", "steps")}
    p.update(nx=NX, particle_cap=1 << 26)
    return p


def main():
    lib = oracle.build_multicore()
    oracle._load(lib).orc_set_threads(os.cpu_count() or 1)
    out = {"what": __doc__.split("\n\n")[0], "nx": NX, "steps": STEPS, "rows": []}
    for idx in ROWS:
        diags = []
        for run in range(SEEDS):
            p = slice_params(idx, run)
            t0 = time.time()
            rec = oracle.Oracle(p, lib_path=lib).step(STEPS)
            e = A.ensemble(rec, p)
            e["seed"] = p["seed"]
            diags.append(e)
            print(f"row {idx} seed {run}: {time.time() - t0:.0f} s", flush=True)
        p0 = slice_params(idx, 0)
        out["rows"].append({"row": idx, "E0": p0["E0"], "gamma_thr": p0["gamma_thr"], "eps_gamma": p0["eps_gamma"],
                            "dt": p0["dt"], "dx": p0["dx"], "diagnostics": diags})
    with open(os.path.join(HERE, "sweep_oracle.json"), "w") as f:
        json.dump(out, f, indent=1, allow_nan=True)


if __name__ == "__main__":
    main()
