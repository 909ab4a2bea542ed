"""The batch autotuner's cache, on the host (no GPU): size-class keys, a
store/lookup round trip through the file, replacement of one key's entry
without touching the others, the last entry of a key winning, and a path
that cannot be written keeping entries in memory for the process."""
import os

import pytest

from paper_2012_05587_gb300 import capi


def test_keys_follow_the_size_class():
    k = capi.cascade_tune_key("fp32", 8192, 2 ** 24, 256)
    assert k == "prec1-nx2^13-np2^24-m2^8"
    # the same class: grid up to the next power of two, particles within a
    # factor sqrt(2), members up to the next power of two
    assert capi.cascade_tune_key("fp32", 5000, int(1.3 * 2 ** 24), 200) == k
    assert capi.cascade_tune_key("fp32", 8193, 2 ** 24, 256) != k
    assert capi.cascade_tune_key("fp64", 8192, 2 ** 24, 256) != k
    assert capi.cascade_tune_key("fp32", 8192, 2 ** 26, 256) != k
    with pytest.raises(capi.CascadeError):
        capi.cascade_tune_key(7, 8192, 1, 1)


def test_store_and_lookup_round_trip(tmp_path):
    path = tmp_path / "sub" / "tune.txt"  # the directories are created on store
    key = capi.cascade_tune_key("fp32", 1024, 10 ** 6, 8)
    assert capi.cascade_tune_cache_lookup(path, key) is None
    capi.cascade_tune_cache_store(path, key, 2, 1, 0, 1024, 0.75)
    other = capi.cascade_tune_key("fp32", 4096, 10 ** 7, 8)
    capi.cascade_tune_cache_store(path, other, 0, 0, 1, 512, 1.5)
    # a new store for the first key replaces its line only
    capi.cascade_tune_cache_store(path, key, 3, 0, 1, 1024, 0.5)
    lines = open(path).read().splitlines()
    assert len(lines) == 2
    assert lines[0].startswith(key + "\t3 0 1 1024\t")
    assert lines[1].startswith(other + "\t0 0 1 512\t")
    assert capi.cascade_tune_cache_lookup(path, key) == {"shape": 3, "stage": 0, "prefetch": 1, "member_cost": 1024}


def test_file_written_by_another_process_is_read(tmp_path):
    """Entries come from the file (not only from this process's memory); of
    several lines for one key the last wins; malformed lines are skipped."""
    path = tmp_path / "tune.txt"
    path.write_text("garbage line\n"
                    "prec1-nx2^10-np2^20-m2^3\t1 1 0 256\t2.0\n"
                    "prec1-nx2^10-np2^20-m2^3\t2 0 1 1024\t1.0\n")
    assert capi.cascade_tune_cache_lookup(path, "prec1-nx2^10-np2^20-m2^3") == \
        {"shape": 2, "stage": 0, "prefetch": 1, "member_cost": 1024}
    assert capi.cascade_tune_cache_lookup(path, "prec1-nx2^11-np2^20-m2^3") is None


def test_unwritable_path_keeps_entries_in_memory(tmp_path):
    blocker = tmp_path / "file"
    blocker.write_text("")
    path = blocker / "tune.txt"  # a directory that cannot exist
    capi.cascade_tune_cache_store(path, "k1", 1, 0, 1, 1024, 3.0)
    assert not os.path.exists(path)
    assert capi.cascade_tune_cache_lookup(path, "k1") == {"shape": 1, "stage": 0, "prefetch": 1, "member_cost": 1024}
    capi.cascade_tune_cache_store(None, "k2", 0, 0, 1, 1024, 3.0)
    assert capi.cascade_tune_cache_lookup(None, "k2")["shape"] == 0


def test_cache_path_honours_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("CASCADE_TUNE_CACHE", str(tmp_path / "x.txt"))
    assert capi.cascade_tune_cache_path() == str(tmp_path / "x.txt")
    monkeypatch.delenv("CASCADE_TUNE_CACHE")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    p = capi.cascade_tune_cache_path()
    assert p.startswith(str(tmp_path) + "/cascade-gb300/batch-tune-") and p.endswith(".txt")
