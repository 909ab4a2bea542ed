"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that ``include/*.h`` declares, and validates parameters on
the host (the model's domain, Section 2-3) before any device work."""
import ctypes
import glob
import os
import re

import pytest

from paper_2012_05587_gb300 import capi, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cascade_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cascade_create", "cascade_step", "cascade_diag", "cascade_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_the_header_layout():
    # cascade_params: 2 int32, 9 double, 1 uint64 ... laid out without padding surprises
    assert ctypes.sizeof(capi.cascade_params) == 4 * 2 + 8 * 9 + 8 * 2 + 4 * 2 + 8 * 2 + 4 * 2
    assert ctypes.sizeof(capi.cascade_diag_t) == 8 * 14


@pytest.mark.parametrize("bad,why", [
    (dict(eps_gamma=1.5), "rest mass"),
    (dict(gamma_thr=10.5, eps_gamma=10.0), "gamma_thr - eps_gamma"),
    (dict(gamma_thr=12.0, eps_gamma=9.0), "2/3"),
    (dict(dt=0.2), "dt"),
    (dict(nx=1), "nx"),
    (dict(l_pp=-1.0), "l_pp"),
    (dict(precision=7), "precision"),
])
def test_host_validation(bad, why):
    p = dict(W.small_cascade(), **bad)
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_footprint(p)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    assert why in str(ei.value)


def test_footprint_and_flight_steps():
    npp, b = capi.cascade_footprint(W.small_cascade())
    assert npp == 20                       # ceil(l_pp / dt) = ceil(1.0 / 0.05)
    npp2, _ = capi.cascade_footprint(dict(W.small_cascade(), l_pp=0.0))
    assert npp2 == 0
    p = W.large_cascade()
    npp3, big = capi.cascade_footprint(p)
    assert npp3 == 20
    # particle storage dominates: 2 species x 12 B x cap in FP32-mixed mode
    assert 2 * 12 * p["particle_cap"] <= big <= 2 * 12 * p["particle_cap"] * 1.5
    _, big64 = capi.cascade_footprint(dict(p, precision="fp64"))
    assert big64 > big


def test_status_strings():
    assert capi.status_string(capi.CASCADE_ERR_CAPACITY) == "particle capacity exceeded"
    assert capi.status_string(12345) == "unknown status"


def test_create_without_device_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_create(W.small_cascade())
    assert ei.value.status == capi.CASCADE_ERR_CUDA


@pytest.mark.parametrize("members,why", [
    ([dict(eps_gamma=1.5)], "member 0: invalid parameters: eps_gamma"),
    ([{}, dict(precision="fp64")], "member 1: precision"),
    ([{}, {}, dict(open_bc=1)], "member 2: batch members are periodic"),
    ([{}, dict(particle_cap=(1 << 30) + 1)], "member 1: batch members hold at most 1073741824 particles"),
])
def test_batch_members_validated_before_device_work(members, why):
    """A batch checks every member on the host (the same domain as a single
    cascade, one precision class, periodic grids, at most 2^30 particles per
    species) before touching a device."""
    ps = [dict(W.small_cascade(precision="fp32"), **m) for m in members]
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_batch_create(ps, 0, 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    assert why in str(ei.value)


def test_batch_slots_validated():
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_batch_create_slots(0, "fp32", 1024, 0, 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_batch_create_slots(4, "fp32", 1, 0, 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG


def test_error_message_describes_the_latest_call_only():
    lib = capi.load()
    with pytest.raises(capi.CascadeError):
        capi.cascade_footprint(dict(W.small_cascade(), eps_gamma=1.5))
    assert b"eps_gamma" in lib.cascade_last_error_message()
    capi.cascade_footprint(W.small_cascade())
    assert lib.cascade_last_error_message() == b""


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "libcascade.so"))
    with pytest.raises(ImportError, match="missing"):
        capi.load()


def test_momentum_words_rule():
    """One FP32 word suffices where half its spacing at the threshold momentum
    is at most 2^-12 of the push per step; otherwise two words are used, and
    asking for one is rejected with a message naming the limit."""
    assert capi.cascade_momentum_words(W.large_cascade()) == 1            # u_thr = 50, push 2.5
    assert capi.cascade_momentum_words(W.small_cascade(precision="fp32")) == 1
    for p in W.precision_sweep() + W.batch_scan(64):
        assert capi.cascade_momentum_words(p) == 1
    # Section 8's threshold, gamma_thr ~ 7.3e7: FP32 spacing 8 against a push of 8
    hot = dict(W.small_cascade(precision="fp32"), E0=1024.0, dt=1.0 / 128.0, gamma_thr=7.3e7, eps_gamma=7.3e5)
    assert capi.cascade_momentum_words(hot) == 2
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_momentum_words(dict(hot, u_words=1))
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG and "2^-12" in str(ei.value)
    # no initial field: the reference push uses gamma_thr / L (co-rotating frame)
    assert capi.cascade_momentum_words(W.corotating()) == 2
    # forcing two words is always allowed; the footprint grows by 4 B per particle and species
    small = W.small_cascade(precision="fp32")
    assert capi.cascade_momentum_words(dict(small, u_words=2)) == 2
    _, b1 = capi.cascade_footprint(small)
    _, b2 = capi.cascade_footprint(dict(small, u_words=2))
    cap4 = (small["particle_cap"] + 3) // 4 * 4
    assert b2 - b1 == 2 * 4 * cap4
    with pytest.raises(capi.CascadeError):
        capi.cascade_momentum_words(dict(small, u_words=3))


def test_batch_rejects_two_word_members():
    ps = [W.small_cascade(precision="fp32"), dict(W.small_cascade(precision="fp32"), u_words=2)]
    with pytest.raises(capi.CascadeError) as ei:
        capi.cascade_batch_create(ps, 0, 0)
    assert ei.value.status == capi.CASCADE_ERR_INVALID_ARG
    assert "member 1: batch members keep one-word FP32 momenta" in str(ei.value)


def test_record_copy_size():
    """A queued record copy moves the control block: the 112-byte record
    with the step's counters and the device error flag (256 B)."""
    assert capi.cascade_record_copy_bytes() == 256
    assert capi.cascade_record_copy_bytes() >= ctypes.sizeof(capi.cascade_diag_t)
