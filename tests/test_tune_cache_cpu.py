"""Tuning results persist across processes through a text file
(pa_tune_cache_save / pa_tune_cache_load); host-only, no device needed."""
import os

from paper_2105_13678_gb300 import _lib


def test_tune_cache_roundtrip(tmp_path):
    L = _lib.lib()
    src = tmp_path / "tune.txt"
    src.write_text("# tuned on a test host\n"
                   "geometry 30402457 9 21 10 4\n"
                   "geometry 60804914 1 22 11 2\n"
                   "backend 30402457 9 2\n"
                   "backend 136279841 8 1\n")
    assert L.pa_tune_cache_load(str(src).encode()) == 4
    out = tmp_path / "saved.txt"
    n = L.pa_tune_cache_save(str(out).encode())
    assert n >= 4
    lines = set(out.read_text().split("\n"))
    for want in ("geometry 30402457 9 21 10 4", "geometry 60804914 1 22 11 2", "backend 30402457 9 2",
                 "backend 136279841 8 1"):
        assert want in lines


def test_tune_cache_rejects_bad_entries(tmp_path):
    L = _lib.lib()
    bad = tmp_path / "bad.txt"
    bad.write_text("geometry 1000 2 21 15 8\n")  # log R beyond the kernels' range
    assert L.pa_tune_cache_load(str(bad).encode()) == _lib.PA_ERR_INVALID
    bad.write_text("backend 30402457 9 7\n")  # no such backend
    assert L.pa_tune_cache_load(str(bad).encode()) == _lib.PA_ERR_INVALID
    bad.write_text("nonsense\n")
    assert L.pa_tune_cache_load(str(bad).encode()) == _lib.PA_ERR_INVALID
    assert L.pa_tune_cache_load(str(tmp_path / "missing.txt").encode()) == _lib.PA_ERR_INVALID
    assert L.pa_tune_cache_save(None) == _lib.PA_ERR_INVALID
    assert not os.path.exists(tmp_path / "missing.txt")
