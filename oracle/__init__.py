"""FP64 CPU oracle of the pair-cascade PIC step (arXiv:2012.05587, Sections 2-3).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library under
``paper_2012_05587_gb300`` never does.  It shares no code with the CUDA path.

The arithmetic lives in ``cascade_oracle.c`` (plain C, double precision, built
with ``-ffp-contract=off``); this module compiles it and marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cascade_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_libs: dict = {}


_LIB_MC = os.path.join(_HERE, "liboracle_mc.so")


def compile_source(src: str, out: str, openmp: bool = False) -> str:
    """Compile an oracle source file into a shared library (gcc, no FMA
    contraction); ``openmp`` gives the multi-core build of the same source."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
        *(["-fopenmp"] if openmp else []), src, "-o", tmp, "-lm",
    ])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def build_multicore(force: bool = False) -> str:
    """Compile the multi-core (OpenMP) build into ``oracle/liboracle_mc.so``;
    it is used only to time the oracle on all host cores."""
    if force or not os.path.exists(_LIB_MC) or os.path.getmtime(_LIB_MC) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_MC, openmp=True)
    return _LIB_MC


SOURCE = _SRC


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ppc", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("n0", ctypes.c_double), ("u_spread", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("E0", ctypes.c_double), ("gamma_thr", ctypes.c_double),
        ("eps_gamma", ctypes.c_double), ("l_pp", ctypes.c_double),
        ("particle_cap", ctypes.c_int64),
        ("j_m", ctypes.c_double), ("rho_gj", ctypes.c_double),
        ("open_bc", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


class OrcDiag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("t", ctypes.c_double), ("E_mean", ctypes.c_double), ("J_mean", ctypes.c_double),
        ("E_absmax", ctypes.c_double), ("U_E", ctypes.c_double), ("U_K", ctypes.c_double),
        ("U_gamma", ctypes.c_double), ("gauss_resid", ctypes.c_double),
        ("n_elec", ctypes.c_int64), ("n_posi", ctypes.c_int64), ("n_photon", ctypes.c_int64),
        ("n_pairs_total", ctypes.c_int64), ("n_emit_multi", ctypes.c_int64),
    ]


DIAG_FIELDS = [f for f, _ in OrcDiag._fields_]


def _load(path: str | None = None):
    with _lock:
        key = path or _LIB
        if key not in _libs:
            lib = ctypes.CDLL(path or build())
            P = ctypes.POINTER
            vp = ctypes.c_void_p
            lib.orc_create.argtypes = [P(OrcParams), P(vp)]
            lib.orc_create_state.argtypes = [P(OrcParams), ctypes.c_int64, vp, vp, vp, vp, vp, P(vp)]
            lib.orc_step.argtypes = [vp, ctypes.c_int32, P(OrcDiag)]
            lib.orc_destroy.argtypes = [vp]
            lib.orc_destroy.restype = None
            for name in ("orc_num_particles", "orc_num_photons", "orc_step_index"):
                getattr(lib, name).argtypes = [vp]
                getattr(lib, name).restype = ctypes.c_int64
            lib.orc_n_pp.argtypes = [vp]
            lib.orc_n_pp.restype = ctypes.c_int32
            lib.orc_get_fields.argtypes = [vp, vp, vp]
            lib.orc_get_fields.restype = None
            lib.orc_get_particles.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_get_particles.restype = None
            lib.orc_get_photons.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_get_photons.restype = None
            lib.orc_diag_now.argtypes = [vp, P(OrcDiag)]
            lib.orc_diag_now.restype = None
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_philox4x32_10.restype = None
            lib.orc_seed_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                             P(ctypes.c_double), P(ctypes.c_double)]
            lib.orc_seed_normals.restype = None
            lib.orc_threads.argtypes = []
            lib.orc_threads.restype = ctypes.c_int32
            lib.orc_set_threads.argtypes = [ctypes.c_int32]
            lib.orc_set_threads.restype = None
            _libs[key] = lib
    return _libs[key]


ERRORS = {-1: "invalid argument", -2: "out of memory", -3: "particle capacity exceeded"}


class OracleError(RuntimeError):
    pass


def _params(p: dict) -> OrcParams:
    return OrcParams(
        nx=int(p["nx"]), ppc=int(p["ppc"]), dx=float(p["dx"]), dt=float(p["dt"]),
        n0=float(p["n0"]), u_spread=float(p["u_spread"]), seed=int(p["seed"]),
        E0=float(p["E0"]), gamma_thr=float(p["gamma_thr"]), eps_gamma=float(p["eps_gamma"]),
        l_pp=float(p["l_pp"]), particle_cap=int(p.get("particle_cap", 1 << 40)),
        j_m=float(p.get("j_m", 0.0)), rho_gj=float(p.get("rho_gj", 0.0)),
        open_bc=int(p.get("open_bc", 0)), pad_=0,
    )


def philox4x32_10(ctr, key, lib_path: str | None = None) -> np.ndarray:
    lib = _load(lib_path)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def seed_normals(seed: int, j: int, lib_path: str | None = None):
    lib = _load(lib_path)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib.orc_seed_normals(seed, j, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


_DIAG_DTYPE = np.dtype([(f, np.int64 if t is ctypes.c_int64 else np.float64) for f, t in OrcDiag._fields_])


def diag_array(recs) -> dict:
    """Per-step diagnostic records -> dict of numpy columns."""
    a = np.frombuffer(recs, dtype=_DIAG_DTYPE)
    return {f: a[f].copy() for f in DIAG_FIELDS}


@dataclass
class Oracle:
    """One cascade advanced by the FP64 oracle (see ``cascade_oracle.c``)."""

    params: dict
    lib_path: str | None = None

    def __post_init__(self):
        self._lib = _load(self.lib_path)
        self._h = ctypes.c_void_p()
        self._p = _params(self.params)
        self._state = self.params.get("_state")
        if self._state is None:
            rc = self._lib.orc_create(ctypes.byref(self._p), ctypes.byref(self._h))
        else:
            st = self._state
            cell = np.ascontiguousarray(st["cell"], dtype=np.int32)
            off = np.ascontiguousarray(st["off"], dtype=np.float64)
            u = np.ascontiguousarray(st["u"], dtype=np.float64)
            q = np.ascontiguousarray(st["q"], dtype=np.int8)
            E = st.get("E")
            E = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
            rc = self._lib.orc_create_state(
                ctypes.byref(self._p), len(cell), cell.ctypes.data, off.ctypes.data,
                u.ctypes.data, q.ctypes.data, None if E is None else E.ctypes.data,
                ctypes.byref(self._h))
        if rc != 0:
            raise OracleError(f"orc_create: {ERRORS.get(rc, rc)}")

    @classmethod
    def from_state(cls, params: dict, cell, off, u, q, E=None, lib_path=None) -> "Oracle":
        p = dict(params)
        p["_state"] = {"cell": cell, "off": off, "u": u, "q": q, "E": E}
        return cls(p, lib_path)

    def step(self, nsteps: int) -> dict:
        recs = (OrcDiag * nsteps)()
        rc = self._lib.orc_step(self._h, nsteps, recs)
        if rc != 0:
            raise OracleError(f"orc_step: {ERRORS.get(rc, rc)}")
        return diag_array(recs)

    def diag_now(self) -> dict:
        d = OrcDiag()
        self._lib.orc_diag_now(self._h, ctypes.byref(d))
        return {f: getattr(d, f) for f in DIAG_FIELDS}

    @property
    def n_pp(self) -> int:
        return self._lib.orc_n_pp(self._h)

    @property
    def num_particles(self) -> int:
        return self._lib.orc_num_particles(self._h)

    @property
    def num_photons(self) -> int:
        return self._lib.orc_num_photons(self._h)

    def fields(self):
        nx = int(self.params["nx"])
        E = np.zeros(nx)
        J = np.zeros(nx)
        self._lib.orc_get_fields(self._h, E.ctypes.data, J.ctypes.data)
        return E, J

    def particles(self) -> dict:
        n = self.num_particles
        cell = np.zeros(n, np.int32)
        off = np.zeros(n)
        u = np.zeros(n)
        q = np.zeros(n, np.int8)
        self._lib.orc_get_particles(self._h, cell.ctypes.data, off.ctypes.data, u.ctypes.data, q.ctypes.data)
        return {"cell": cell, "off": off, "u": u, "q": q}

    def photons(self) -> dict:
        n = self.num_photons
        cs = np.zeros(n, np.int64)
        cell = np.zeros(n, np.int32)
        off = np.zeros(n)
        d = np.zeros(n, np.int8)
        self._lib.orc_get_photons(self._h, cs.ctypes.data, cell.ctypes.data, off.ctypes.data, d.ctypes.data)
        return {"conv_step": cs, "cell": cell, "off": off, "dir": d}

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
