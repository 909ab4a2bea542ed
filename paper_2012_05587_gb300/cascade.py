"""A cascade handle with Python lifetime management (thin wrapper over the C ABI)."""
from __future__ import annotations

import numpy as np

from . import capi


def _torch_stream() -> int:
    import torch

    return int(torch.cuda.current_stream().cuda_stream)


class Cascade:
    """One cascade resident on the current CUDA device.

    ``params`` holds the fields of ``cascade_params``; ``state`` optionally
    gives explicit particles (``{"elec": {...}, "posi": {...}, "E": array}``).
    Device memory comes from PyTorch's caching allocator and work runs on
    PyTorch's current stream unless ``stream`` (a cudaStream_t as int) is given.
    """

    def __init__(self, params: dict, state: dict | None = None, stream: int | None = None,
                 torch_memory: bool = True):
        if torch_memory:
            capi.use_torch_allocator()
        self.params = dict(params)
        self.nx = int(params["nx"])
        self.stream = _torch_stream() if stream is None else int(stream)
        if state is None:
            self.h = capi.cascade_create(self.params, self.stream)
        else:
            self.h = capi.cascade_create_from_state(self.params, state["elec"], state["posi"], state.get("E"),
                                                    self.stream)

    def step(self, nsteps: int) -> None:
        capi.cascade_step(self.h, nsteps)

    def sync(self) -> None:
        capi.cascade_sync(self.h)

    def diag(self, max_records: int = 1 << 16) -> dict:
        return capi.cascade_diag(self.h, max_records)

    def record_enqueue(self) -> None:
        """Queue a copy of the newest step's record to the host (no wait)."""
        capi.cascade_record_enqueue(self.h)

    def record_poll(self, max_records: int = 64, wait: bool = False) -> dict:
        """The queued records that have landed, oldest first."""
        return capi.cascade_record_poll(self.h, max_records, wait)

    def fields(self):
        _, E, J = capi.cascade_diag(self.h, 0, self.nx, fields=True)
        return E, J

    def gauss(self) -> float:
        return capi.cascade_gauss(self.h)

    def set_gauss_every(self, every: int) -> None:
        capi.cascade_set_gauss_every(self.h, every)

    def counts(self) -> dict:
        return capi.cascade_counts(self.h)

    def particles(self, species: int) -> dict:
        c = self.counts()
        n = c["n_elec"] if species == 0 else c["n_posi"]
        return capi.cascade_particles(self.h, species, n)

    def histogram(self, species: int, quantity: str, nbins: int, lo: float, hi: float) -> np.ndarray:
        q = {"u": capi.HIST_U, "gamma": capi.HIST_GAMMA, "x": capi.HIST_X}[quantity]
        return capi.cascade_histogram(self.h, species, q, nbins, lo, hi)

    def close(self) -> None:
        if getattr(self, "h", None):
            capi.cascade_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def diag_to_arrays(rec: dict) -> dict:
    return {k: np.asarray(v) for k, v in rec.items()}


class CascadeBatch:
    """Many cascades advanced together (one launch per kernel per step).

    Either ``CascadeBatch(params_list)`` (every member in its initial state,
    advanced with ``step``), or ``CascadeBatch(slots=..., precision=...,
    max_nx=...)`` for admission-driven serving (``admit``/``run``/``poll``).
    """

    def __init__(self, params: list | None = None, *, slots: int = 0, precision="fp32", max_nx: int = 0,
                 hbm_budget: int = 0, stream: int | None = None, torch_memory: bool = True):
        if torch_memory:
            capi.use_torch_allocator()
        self.stream = _torch_stream() if stream is None else int(stream)
        self.params = {}
        if params is not None:
            self.b = capi.cascade_batch_create(params, hbm_budget, self.stream)
            self.params = {i: dict(p) for i, p in enumerate(params)}
        else:
            self.b = capi.cascade_batch_create_slots(slots, precision, max_nx, hbm_budget, self.stream)

    def admit(self, params: dict, nsteps: int) -> int:
        slot = capi.cascade_batch_admit(self.b, params, nsteps)
        self.params[slot] = dict(params)
        return slot

    def step(self, nsteps_each) -> None:
        capi.cascade_batch_step(self.b, nsteps_each)

    def run(self, nsteps: int) -> None:
        capi.cascade_batch_run(self.b, nsteps)

    def poll(self, wait: bool = False, max_n: int = 4096) -> list:
        return capi.cascade_batch_poll(self.b, max_n, wait)

    def diag(self, slot: int, max_records: int = 1 << 16) -> dict:
        return capi.cascade_batch_diag(self.b, slot, max_records)

    def fields(self, slot: int):
        _, E, J = capi.cascade_batch_diag(self.b, slot, 0, int(self.params[slot]["nx"]), fields=True)
        return E, J

    def counts(self, slot: int) -> dict:
        return capi.cascade_batch_counts(self.b, slot)

    def release(self, slot: int) -> None:
        capi.cascade_batch_release(self.b, slot)
        self.params.pop(slot, None)

    def info(self) -> dict:
        return capi.cascade_batch_info(self.b)

    def variant(self) -> dict:
        return capi.cascade_batch_get_variant(self.b)

    def set_variant(self, shape: int, stage: int, prefetch: int, member_cost: int = 1024) -> None:
        capi.cascade_batch_set_variant(self.b, shape, stage, prefetch, member_cost)

    def tune_next(self, rounds: int = 4, use_cache: bool = True, warmup: int | None = None) -> None:
        if warmup is not None:
            capi.cascade_batch_tune_warmup(self.b, warmup)
        capi.cascade_batch_tune_next(self.b, rounds, use_cache)

    def tuning_report(self) -> list:
        return capi.cascade_batch_tuning_report(self.b)

    def close(self) -> None:
        if getattr(self, "b", None):
            capi.cascade_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
