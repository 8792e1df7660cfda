"""The C-ABI library loads on a CPU-only host and exports every entry point that include/*.h
declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(zm\w*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("zm_create", "zm_velocity", "zm_step", "zm_destroy", "zm_set_state", "zm_get_state",
                 "zm_set_stream", "zm_sync", "zm_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2406_05490_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # status strings are pure host code
    lib.zm_error_string.restype = ctypes.c_char_p
    assert lib.zm_error_string(0) == b"ok"
    assert lib.zm_error_string(-5) == b"unsupported configuration"
    # the checked build (same sources, ZM_CHECKS=1) exports the same entry points and says so
    chk = ctypes.CDLL(build.LIB_CHECKED)
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    assert lib.zm_checked_build() == 0 and chk.zm_checked_build() == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2406_05490_gb300 import zm
    monkeypatch.setattr(zm, "_lib", None)
    monkeypatch.setattr(zm, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(zm.ZMError):
        zm.load()


def test_binding_resolves_every_entry_point():
    """The ctypes binding declares a signature for every exported entry point it wraps, and
    every name it wraps is declared in include/zm.h (no compute call is made)."""
    from paper_2406_05490_gb300 import build, zm
    build.build()
    zm._lib = None
    lib = zm.load()
    declared = set(declared_functions())
    import inspect
    for name in dir(zm):
        if name.startswith("zm_") and inspect.isfunction(getattr(zm, name)):
            assert name in declared, name
            assert hasattr(lib, name)


def test_binding_constants_match_header():
    """Every integer #define of include/zm.h (status codes, order and precision flags, kernel
    classes, request states) has the same value in the Python binding."""
    from paper_2406_05490_gb300 import zm
    src = open(os.path.join(ROOT, "include", "zm.h")).read()
    found = 0
    for m in re.finditer(r"^#define\s+(ZM_\w+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))\)?", src, flags=re.M):
        name, value = m.group(1), int(m.group(2), 0)
        assert hasattr(zm, name), name
        assert getattr(zm, name) == value, (name, getattr(zm, name), value)
        found += 1
    assert found >= 24
