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

    def fields(self):
        _, E, J = capi.cascade_diag(self.h, 0, self.nx, fields=True)
        return E, J

    def gauss(self) -> float:
        return capi.cascade_gauss(self.h)

    def counts(self) -> dict:
        return capi.cascade_counts(self.h)

    def particles(self, species: int) -> dict:
        c = self.counts()
        n = c["n_elec"] if species == 0 else c["n_posi"]
        return capi.cascade_particles(self.h, species, n)

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
