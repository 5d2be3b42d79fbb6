"""The C ABI library builds, loads without a GPU and exports every entry
point include/svt.h declares; host-side argument checks need no device."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "svt.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(svt_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_0917_gb300 import binding
    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_1312_0917_gb300 import binding
    assert set(binding.SIGNATURES) == set(names)


def test_strerror_and_null_checks(lib):
    from paper_1312_0917_gb300 import binding as B
    assert lib.svt_strerror(B.OK) == b"ok"
    assert lib.svt_strerror(B.E_TIMEOUT) == b"device-side wait timed out"
    assert lib.svt_create(None, 0, None) == B.E_INVAL
    assert lib.svt_fit_events(None, 1, None) == B.E_INVAL
    assert lib.svt_unpack(None, None, 0, None) == B.E_INVAL
    n = C.c_size_t()
    assert lib.svt_get_tracks(None, None, 0, C.byref(n), None) == B.E_INVAL
    assert lib.svt_last_launch_count(None) == 0
    assert lib.svt_server_create(None, 0, None, None, 0, 0) == B.E_INVAL
    assert lib.svt_server_submit(None, None, 0, None) == B.E_INVAL
    assert lib.svt_set_launch(None, None) == B.E_INVAL and lib.svt_get_launch(None, None) == B.E_INVAL


def test_struct_layouts():
    from paper_1312_0917_gb300 import binding as B
    assert B.CONST_DTYPE.itemsize == 96
    assert B.TRACK_DTYPE.itemsize == 40 and B.TRACK_DTYPE.fields["chi2"][1] == 24
    assert B.ROAD_DTYPE.itemsize == 100 and B.ROAD_DTYPE.fields["coord"][1] == 20
    assert C.sizeof(B.Limits) == 40 and C.sizeof(B.Stats) == 104
    assert C.sizeof(B.ServerConfig) == 56 and C.sizeof(B.ServerResult) == 48
    assert C.sizeof(B.Launch) == 20 and C.sizeof(B.TunePoint) == 24


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_1312_0917_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        B.lib()
