"""ctypes binding of the C ABI in ``include/cascade.h`` (argument marshalling only).

Every entry point keeps its C name.  All compute runs in ``libcascade.so``;
this module only converts Python values to C structs and pointers.  Loading
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcascade.so")

CASCADE_OK = 0
CASCADE_ERR_INVALID_ARG = -1
CASCADE_ERR_OOM = -2
CASCADE_ERR_CAPACITY = -3
CASCADE_ERR_CUDA = -4
CASCADE_ERR_TIMEOUT = -5
CASCADE_ERR_UNIMPLEMENTED = -6
CASCADE_ERR_PHOTON_CAPACITY = -7
CASCADE_ERR_BUSY = -8
CASCADE_ERR_NONFINITE = -9

CASCADE_FP64 = 0
CASCADE_FP32_MIXED = 1
CASCADE_FP32_MIXED_FINE = 2


class cascade_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ppc", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("n0", ctypes.c_double), ("u_spread", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("E0", ctypes.c_double), ("gamma_thr", ctypes.c_double),
        ("eps_gamma", ctypes.c_double), ("l_pp", ctypes.c_double),
        ("particle_cap", ctypes.c_int64), ("photon_cap", ctypes.c_int64),
        ("precision", ctypes.c_int32), ("diag_ring", ctypes.c_int32),
        ("j_m", ctypes.c_double), ("rho_gj", ctypes.c_double),
        ("open_bc", ctypes.c_int32), ("u_words", ctypes.c_int32),
    ]


class cascade_diag_t(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("t", ctypes.c_double), ("E_mean", ctypes.c_double), ("J_mean", ctypes.c_double),
        ("E_absmax", ctypes.c_double), ("U_E", ctypes.c_double), ("U_K", ctypes.c_double),
        ("U_gamma", ctypes.c_double), ("gauss_resid", ctypes.c_double),
        ("n_elec", ctypes.c_int64), ("n_posi", ctypes.c_int64), ("n_photon", ctypes.c_int64),
        ("n_pairs_total", ctypes.c_int64), ("n_emit_multi", ctypes.c_int64),
    ]


DIAG_FIELDS = [f for f, _ in cascade_diag_t._fields_]
DIAG_DTYPE = np.dtype([(f, np.int64 if t is ctypes.c_int64 else np.float64) for f, t in cascade_diag_t._fields_])

class cascade_batch_variant(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("stage", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("member_cost", ctypes.c_int32)]


VARIANT_SOURCES = {0: "default", 1: "cached", 2: "tuned", 3: "forced"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


class CascadeError(RuntimeError):
    def __init__(self, where: str, status: int, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def load() -> ctypes.CDLL:
    """Load libcascade.so (built by ``paper_2012_05587_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2012_05587_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "cascade_set_allocator": ([ALLOC_FN, FREE_FN, vp], ctypes.c_int),
            "cascade_create": ([P(cascade_params), vp, P(vp)], ctypes.c_int),
            "cascade_create_from_state": ([P(cascade_params), i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, P(vp)],
                                          ctypes.c_int),
            "cascade_create_from_state_f32": ([P(cascade_params), i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, P(vp)],
                                              ctypes.c_int),
            "cascade_step": ([vp, i32], ctypes.c_int),
            "cascade_sync": ([vp], ctypes.c_int),
            "cascade_diag": ([vp, vp, i32, P(i32), vp, vp], ctypes.c_int),
            "cascade_record_enqueue": ([vp], ctypes.c_int),
            "cascade_record_poll": ([vp, vp, i32, i32, P(i32)], ctypes.c_int),
            "cascade_record_copy_bytes": ([], ctypes.c_int32),
            "cascade_gauss": ([vp, P(f64)], ctypes.c_int),
            "cascade_set_gauss_every": ([vp, i32], ctypes.c_int),
            "cascade_counts": ([vp, P(i64), P(i64), P(i64), P(i64)], ctypes.c_int),
            "cascade_particles": ([vp, i32, i64, vp, vp, vp, P(i64)], ctypes.c_int),
            "cascade_histogram": ([vp, i32, i32, i32, f64, f64, vp], ctypes.c_int),
            "cascade_destroy": ([vp], ctypes.c_int),
            "cascade_footprint": ([P(cascade_params), P(i32), P(ctypes.c_size_t)], ctypes.c_int),
            "cascade_momentum_words": ([P(cascade_params), P(i32)], ctypes.c_int),
            "cascade_set_timing": ([vp, i32], ctypes.c_int),
            "cascade_timing": ([vp, P(f64), P(i64), P(i64)], ctypes.c_int),
            "cascade_gauss_noalloc": ([i32, f64, f64, f64, i32, i32, i64, vp, vp, i64, vp, vp, vp, P(f64), vp],
                                      ctypes.c_int),
            "cascade_batch_create_slots": ([i32, i32, i32, ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
            "cascade_batch_create": ([P(cascade_params), i32, ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
            "cascade_batch_admit": ([vp, P(cascade_params), i32, P(i32)], ctypes.c_int),
            "cascade_batch_step": ([vp, vp], ctypes.c_int),
            "cascade_batch_run": ([vp, i32], ctypes.c_int),
            "cascade_batch_poll": ([vp, vp, i32, P(i32), i32], ctypes.c_int),
            "cascade_batch_diag": ([vp, i32, vp, i32, P(i32), vp, vp], ctypes.c_int),
            "cascade_batch_counts": ([vp, i32, P(i64), P(i64), P(i64), P(i64)], ctypes.c_int),
            "cascade_batch_release": ([vp, i32], ctypes.c_int),
            "cascade_batch_info": ([vp, P(i32), P(i32), P(ctypes.c_size_t)], ctypes.c_int),
            "cascade_batch_destroy": ([vp], ctypes.c_int),
            "cascade_batch_set_timing": ([vp, i32], ctypes.c_int),
            "cascade_batch_set_variant": ([vp, P(cascade_batch_variant)], ctypes.c_int),
            "cascade_batch_get_variant": ([vp, P(cascade_batch_variant), P(i32), P(f64)], ctypes.c_int),
            "cascade_batch_tune_next": ([vp, i32, i32], ctypes.c_int),
            "cascade_batch_tune_warmup": ([vp, i64], ctypes.c_int),
            "cascade_batch_tuning_report": ([vp, P(cascade_batch_variant), P(f64), i32, P(i32)], ctypes.c_int),
            "cascade_tune_key": ([i32, i32, i64, i32, ctypes.c_char_p, i32], ctypes.c_int),
            "cascade_tune_cache_lookup": ([ctypes.c_char_p, ctypes.c_char_p, P(cascade_batch_variant), P(i32)],
                                          ctypes.c_int),
            "cascade_tune_cache_store": ([ctypes.c_char_p, ctypes.c_char_p, P(cascade_batch_variant), f64],
                                         ctypes.c_int),
            "cascade_tune_cache_path": ([], ctypes.c_char_p),
            "cascade_batch_timing": ([vp, P(f64), P(i64), P(i64)], ctypes.c_int),
            "cascade_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "cascade_last_error_message": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().cascade_status_string(status).decode()


def last_error_message() -> str:
    return load().cascade_last_error_message().decode()


def check(where: str, status: int) -> None:
    if status != CASCADE_OK:
        raise CascadeError(where, status, last_error_message())


def make_params(p: dict) -> cascade_params:
    prec = p.get("precision", CASCADE_FP64)
    if isinstance(prec, str):
        prec = {"fp64": CASCADE_FP64, "fp32": CASCADE_FP32_MIXED, "fp32_mixed": CASCADE_FP32_MIXED,
                "fp32_fine": CASCADE_FP32_MIXED_FINE}[prec]
    return cascade_params(
        nx=int(p["nx"]), ppc=int(p["ppc"]), dx=float(p["dx"]), dt=float(p["dt"]),
        n0=float(p["n0"]), u_spread=float(p["u_spread"]), seed=int(p["seed"]),
        E0=float(p["E0"]), gamma_thr=float(p["gamma_thr"]), eps_gamma=float(p["eps_gamma"]),
        l_pp=float(p["l_pp"]), particle_cap=int(p.get("particle_cap", 1 << 20)),
        photon_cap=int(p.get("photon_cap", 0)), precision=int(prec),
        diag_ring=int(p.get("diag_ring", 0)),
        j_m=float(p.get("j_m", 0.0)), rho_gj=float(p.get("rho_gj", 0.0)),
        open_bc=int(p.get("open_bc", 0)), u_words=int(p.get("u_words", 0)),
    )


# --- device memory from PyTorch's caching allocator -----------------------------

_torch_hooks = None


def use_torch_allocator() -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    import torch

    if _torch_hooks is not None:
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    check("cascade_set_allocator", load().cascade_set_allocator(hooks[0], hooks[1], None))
    _torch_hooks = hooks


# --- the entry points ---------------------------------------------------------------

def _ptr(a):
    return None if a is None else a.ctypes.data


def cascade_create(params: dict, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    cp = make_params(params)
    check("cascade_create", load().cascade_create(ctypes.byref(cp), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def cascade_create_from_state(params: dict, elec: dict, posi: dict, E=None, stream: int = 0) -> ctypes.c_void_p:
    """Explicit state from host arrays: FP32 offsets and momenta in both
    species go through cascade_create_from_state_f32, anything else through
    cascade_create_from_state (FP64)."""
    f32 = all(np.asarray(s[k]).dtype == np.float32 for s in (elec, posi) for k in ("off", "u"))
    real = np.float32 if f32 else np.float64

    def arrays(s):
        return (np.ascontiguousarray(s["cell"], np.int32), np.ascontiguousarray(s["off"], real),
                np.ascontiguousarray(s["u"], real))
    ce, oe, ue = arrays(elec)
    cp_, op, up = arrays(posi)
    E = None if E is None else np.ascontiguousarray(E, np.float64)
    h = ctypes.c_void_p()
    cp = make_params(params)
    name = "cascade_create_from_state_f32" if f32 else "cascade_create_from_state"
    check(name, getattr(load(), name)(
        ctypes.byref(cp), len(ce), _ptr(ce), _ptr(oe), _ptr(ue), len(cp_), _ptr(cp_), _ptr(op), _ptr(up),
        _ptr(E), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def cascade_step(h, nsteps: int) -> None:
    check("cascade_step", load().cascade_step(h, int(nsteps)))


def cascade_sync(h) -> None:
    check("cascade_sync", load().cascade_sync(h))


def cascade_diag(h, max_records: int, nx: int | None = None, fields: bool = False):
    """Newest per-step records (oldest first) as numpy columns; with
    ``fields=True`` also the current E and the last J (nx values each)."""
    buf = (cascade_diag_t * max(max_records, 1))()
    n = ctypes.c_int32()
    E = J = None
    if fields:
        E = np.zeros(nx)
        J = np.zeros(nx)
    check("cascade_diag", load().cascade_diag(h, buf, int(max_records), ctypes.byref(n), _ptr(E), _ptr(J)))
    a = np.frombuffer(buf, dtype=DIAG_DTYPE)[: n.value]
    rec = {f: a[f].copy() for f in DIAG_FIELDS}
    return (rec, E, J) if fields else rec


def cascade_record_enqueue(h) -> None:
    check("cascade_record_enqueue", load().cascade_record_enqueue(h))


def cascade_record_copy_bytes() -> int:
    return int(load().cascade_record_copy_bytes())


def cascade_record_poll(h, max_records: int = 64, wait: bool = False) -> dict:
    """Queued per-step records that have landed (all of them, waiting, with
    ``wait``), oldest first, as numpy columns."""
    buf = (cascade_diag_t * max(max_records, 1))()
    n = ctypes.c_int32()
    check("cascade_record_poll", load().cascade_record_poll(h, buf, int(max_records), int(bool(wait)),
                                                            ctypes.byref(n)))
    a = np.frombuffer(buf, dtype=DIAG_DTYPE)[: n.value]
    return {f: a[f].copy() for f in DIAG_FIELDS}


def cascade_gauss(h) -> float:
    r = ctypes.c_double()
    check("cascade_gauss", load().cascade_gauss(h, ctypes.byref(r)))
    return r.value


def cascade_set_gauss_every(h, every: int) -> None:
    check("cascade_set_gauss_every", load().cascade_set_gauss_every(h, int(every)))


def cascade_counts(h) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    check("cascade_counts", load().cascade_counts(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(("n_elec", "n_posi", "n_photon", "step"), (x.value for x in v)))


def cascade_particles(h, species: int, max_n: int) -> dict:
    cell = np.zeros(max_n, np.int32)
    off = np.zeros(max_n)
    u = np.zeros(max_n)
    n = ctypes.c_int64()
    check("cascade_particles", load().cascade_particles(h, int(species), int(max_n), _ptr(cell), _ptr(off),
                                                        _ptr(u), ctypes.byref(n)))
    k = n.value
    return {"cell": cell[:k], "off": off[:k], "u": u[:k]}


HIST_U, HIST_GAMMA, HIST_X = 0, 1, 2


def cascade_histogram(h, species: int, quantity: int, nbins: int, lo: float, hi: float) -> np.ndarray:
    out = np.zeros(nbins, np.int64)
    check("cascade_histogram", load().cascade_histogram(h, int(species), int(quantity), int(nbins), float(lo),
                                                        float(hi), out.ctypes.data))
    return out


def cascade_destroy(h) -> None:
    if h:
        check("cascade_destroy", load().cascade_destroy(h))


def cascade_set_timing(h, enable: bool) -> None:
    check("cascade_set_timing", load().cascade_set_timing(h, 1 if enable else 0))


def cascade_timing(h) -> dict:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    k = ctypes.c_int64()
    check("cascade_timing", load().cascade_timing(h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
    return {"particle_kernel_ms": ms.value, "particle_kernel_launches": n.value, "kernels_launched": k.value}


def cascade_gauss_noalloc(nx: int, dx: float, w: float, precision: int, n_elec: int, cell_e: int, off_e: int,
                          n_posi: int, cell_p: int, off_p: int, E: int, stream: int = 0, rho_gj: float = 0.0,
                          open_bc: int = 0) -> float:
    """Gauss residual of caller-held DEVICE buffers (pointers as ints); the
    library allocates nothing for this call."""
    r = ctypes.c_double()
    check("cascade_gauss_noalloc", load().cascade_gauss_noalloc(
        int(nx), float(dx), float(w), float(rho_gj), int(open_bc), int(precision), int(n_elec),
        ctypes.c_void_p(cell_e), ctypes.c_void_p(off_e), int(n_posi), ctypes.c_void_p(cell_p),
        ctypes.c_void_p(off_p), ctypes.c_void_p(E), ctypes.byref(r), ctypes.c_void_p(stream)))
    return r.value


def cascade_footprint(params: dict):
    npp = ctypes.c_int32()
    b = ctypes.c_size_t()
    cp = make_params(params)
    check("cascade_footprint", load().cascade_footprint(ctypes.byref(cp), ctypes.byref(npp), ctypes.byref(b)))
    return npp.value, b.value


def cascade_momentum_words(params: dict) -> int:
    w = ctypes.c_int32()
    cp = make_params(params)
    check("cascade_momentum_words", load().cascade_momentum_words(ctypes.byref(cp), ctypes.byref(w)))
    return w.value


# --- batches ---------------------------------------------------------------------------

def _prec_code(prec) -> int:
    if isinstance(prec, str):
        return {"fp64": CASCADE_FP64, "fp32": CASCADE_FP32_MIXED, "fp32_mixed": CASCADE_FP32_MIXED,
                "fp32_fine": CASCADE_FP32_MIXED_FINE}[prec]
    return int(prec)


def cascade_batch_create_slots(max_slots: int, precision, max_nx: int, hbm_budget: int = 0,
                               stream: int = 0) -> ctypes.c_void_p:
    b = ctypes.c_void_p()
    check("cascade_batch_create_slots", load().cascade_batch_create_slots(
        int(max_slots), _prec_code(precision), int(max_nx), int(hbm_budget), ctypes.c_void_p(stream),
        ctypes.byref(b)))
    return b


def cascade_batch_create(params: list, hbm_budget: int = 0, stream: int = 0) -> ctypes.c_void_p:
    arr = (cascade_params * len(params))(*[make_params(p) for p in params])
    b = ctypes.c_void_p()
    check("cascade_batch_create", load().cascade_batch_create(arr, len(params), int(hbm_budget),
                                                              ctypes.c_void_p(stream), ctypes.byref(b)))
    return b


def cascade_batch_admit(b, params: dict, nsteps: int) -> int:
    slot = ctypes.c_int32()
    cp = make_params(params)
    check("cascade_batch_admit", load().cascade_batch_admit(b, ctypes.byref(cp), int(nsteps), ctypes.byref(slot)))
    return slot.value


def cascade_batch_step(b, nsteps_each) -> None:
    a = np.ascontiguousarray(nsteps_each, dtype=np.int32)
    check("cascade_batch_step", load().cascade_batch_step(b, a.ctypes.data))


def cascade_batch_run(b, nsteps: int) -> None:
    check("cascade_batch_run", load().cascade_batch_run(b, int(nsteps)))


def cascade_batch_poll(b, max_n: int, wait: bool = False) -> list:
    buf = np.zeros(max(max_n, 1), np.int32)
    n = ctypes.c_int32()
    check("cascade_batch_poll", load().cascade_batch_poll(b, buf.ctypes.data, int(max_n), ctypes.byref(n),
                                                          1 if wait else 0))
    return [int(x) for x in buf[: n.value]]


def cascade_batch_diag(b, slot: int, max_records: int, nx: int | None = None, fields: bool = False):
    buf = (cascade_diag_t * max(max_records, 1))()
    n = ctypes.c_int32()
    E = J = None
    if fields:
        E = np.zeros(nx)
        J = np.zeros(nx)
    check("cascade_batch_diag", load().cascade_batch_diag(b, int(slot), buf, int(max_records), ctypes.byref(n),
                                                          _ptr(E), _ptr(J)))
    a = np.frombuffer(buf, dtype=DIAG_DTYPE)[: n.value]
    rec = {f: a[f].copy() for f in DIAG_FIELDS}
    return (rec, E, J) if fields else rec


def cascade_batch_counts(b, slot: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    check("cascade_batch_counts", load().cascade_batch_counts(b, int(slot), *[ctypes.byref(x) for x in v]))
    return dict(zip(("n_elec", "n_posi", "n_photon", "step"), (x.value for x in v)))


def cascade_batch_release(b, slot: int) -> None:
    check("cascade_batch_release", load().cascade_batch_release(b, int(slot)))


def cascade_batch_info(b) -> dict:
    s, o, u = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    check("cascade_batch_info", load().cascade_batch_info(b, ctypes.byref(s), ctypes.byref(o), ctypes.byref(u)))
    return {"slots": s.value, "occupied": o.value, "bytes": u.value}


def cascade_batch_set_timing(b, enable: bool) -> None:
    check("cascade_batch_set_timing", load().cascade_batch_set_timing(b, 1 if enable else 0))


def cascade_batch_timing(b) -> dict:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    k = ctypes.c_int64()
    check("cascade_batch_timing", load().cascade_batch_timing(b, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
    return {"particle_kernel_ms": ms.value, "particle_kernel_launches": n.value, "kernels_launched": k.value}


def _variant_dict(v) -> dict:
    return {"shape": v.shape, "stage": v.stage, "prefetch": v.prefetch, "member_cost": v.member_cost}


def cascade_batch_set_variant(b, shape: int, stage: int, prefetch: int, member_cost: int = 1024) -> None:
    v = cascade_batch_variant(shape, stage, prefetch, member_cost)
    check("cascade_batch_set_variant", load().cascade_batch_set_variant(b, ctypes.byref(v)))


def cascade_batch_get_variant(b) -> dict:
    v = cascade_batch_variant()
    src = ctypes.c_int32()
    ns = ctypes.c_double()
    check("cascade_batch_get_variant", load().cascade_batch_get_variant(b, ctypes.byref(v), ctypes.byref(src),
                                                                        ctypes.byref(ns)))
    return dict(_variant_dict(v), source=VARIANT_SOURCES.get(src.value, src.value), ns_per_unit=ns.value)


def cascade_batch_tune_next(b, rounds: int = 4, use_cache: bool = True) -> None:
    check("cascade_batch_tune_next", load().cascade_batch_tune_next(b, int(rounds), 1 if use_cache else 0))


def cascade_batch_tune_warmup(b, steps: int) -> None:
    check("cascade_batch_tune_warmup", load().cascade_batch_tune_warmup(b, int(steps)))


def cascade_batch_tuning_report(b) -> list:
    cands = (cascade_batch_variant * 16)()
    ns = (ctypes.c_double * 16)()
    n = ctypes.c_int32()
    check("cascade_batch_tuning_report", load().cascade_batch_tuning_report(b, cands, ns, 16, ctypes.byref(n)))
    return [dict(_variant_dict(cands[i]), ns_per_unit=ns[i]) for i in range(n.value)]


def cascade_tune_key(precision, max_nx: int, particles: int, members: int) -> str:
    buf = ctypes.create_string_buffer(128)
    check("cascade_tune_key", load().cascade_tune_key(_prec_code(precision), int(max_nx), int(particles),
                                                      int(members), buf, len(buf)))
    return buf.value.decode()


def cascade_tune_cache_lookup(path, key: str):
    v = cascade_batch_variant()
    found = ctypes.c_int32()
    check("cascade_tune_cache_lookup", load().cascade_tune_cache_lookup(
        None if path is None else str(path).encode(), key.encode(), ctypes.byref(v), ctypes.byref(found)))
    return _variant_dict(v) if found.value else None


def cascade_tune_cache_store(path, key: str, shape: int, stage: int, prefetch: int, member_cost: int,
                             ns_per_unit: float) -> None:
    v = cascade_batch_variant(shape, stage, prefetch, member_cost)
    check("cascade_tune_cache_store", load().cascade_tune_cache_store(
        None if path is None else str(path).encode(), key.encode(), ctypes.byref(v), float(ns_per_unit)))


def cascade_tune_cache_path() -> str:
    return load().cascade_tune_cache_path().decode()


def cascade_batch_destroy(b) -> None:
    if b:
        check("cascade_batch_destroy", load().cascade_batch_destroy(b))
