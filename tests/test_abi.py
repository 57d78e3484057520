"""The C-ABI library: it builds, loads, exports every declared entry point, and
its host-side argument checks work -- no GPU needed (no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    L = R.lib()
    declared = _native.header_functions()
    assert "raster_contract" in declared and "raster_agglomerate" in declared
    missing = [f for f in declared if not hasattr(L, f)]
    assert not missing, missing


def test_every_declaration_cites_its_source_or_says_it_has_none():
    """The comment just above each entry point names the paper passage that
    defines the operation, or says that the paper has no counterpart."""
    cite = re.compile(r"Alg\. \d|Sect\. \d|App\. [A-D]|no counterpart in the paper|paper has no counterpart", re.I)
    for fn in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", fn)).read()
        for m in re.finditer(r"^(?:const\s+)?[a-z_0-9]+\s*\**\s*(raster_[a-z0-9_]+)\s*\(", src, flags=re.M):
            before = src[:m.start()]
            end = before.rstrip().rfind("*/")
            assert end >= 0 and before.rstrip().endswith("*/"), f"{m.group(1)} has no comment"
            start = before.rfind("/*", 0, end)
            comment = " ".join(before[start:end].replace("*", " ").split())
            assert cite.search(comment), f"{m.group(1)}: {comment[:80]}"


def test_strerror_and_argument_checks_without_gpu():
    L = R.lib()
    assert L.raster_strerror(0) == b"ok"
    assert b"range" in L.raster_strerror(_native.E_RANGE)
    h = ctypes.c_void_p()
    # invalid tau / mu / precision are rejected before any device work
    assert L.raster_create(2.0, 0, 4, ctypes.byref(h)) == _native.E_ARG
    assert L.raster_create(2.0, 5, 0, ctypes.byref(h)) == _native.E_ARG
    assert L.raster_create(float("nan"), 5, 4, ctypes.byref(h)) == _native.E_ARG
    assert L.raster_create(-400.0, 5, 4, ctypes.byref(h)) == _native.E_ARG  # 10^-400 is not a normal double
    assert L.raster_create(2.0, 5, 4, None) == _native.E_ARG
    assert L.raster_contract(None, None, 0, None) == _native.E_ARG
    assert L.raster_agglomerate(None, None) == _native.E_ARG
    assert L.raster_destroy(None) == _native.E_ARG


def test_binding_raises_when_library_missing(tmp_path, monkeypatch):
    """No CPU fallback: a missing library is a loud error."""
    import importlib
    from paper_1907_03620_gb300 import builder
    monkeypatch.setattr(builder, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(builder, "up_to_date", lambda: True)
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(OSError):
        _native.lib()
